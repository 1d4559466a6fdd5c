#!/usr/bin/env python
"""Throughput benchmark: particle-element passes per second of the spin-orbit
tracker on the RHIC-scale synthetic ring (108 FODO cells, 432 sector bends,
matrix-kick quadrupoles, drift-kick sextupoles, two Siberian snakes; 1514
elements per turn), 10^5 Gaussian protons per GPU, G*gamma0 = 45.5,
Romberg order 2.

One step = one turn of the whole ensemble through the ring (every element,
all slices, the spin step included).  `value` is measured with the particle
state resident in HBM; `e2e` includes, every step, the upload of the state
from pinned host memory through the C ABI and the download of spins, orbit
and lost flags.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
    python bench.py --impl reference ...     # the CPU oracle, timed on host cores

For N > 1 (torchrun) each rank tracks its own 10^5 particles (weak scaling,
no data-path collective); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

WORKLOAD = "rhic_like_1e5"
L2_BYTES = 126 * 1024 * 1024

# Algorithmic work per particle-element pass of this workload (both G gamma0;
# slices max(4, 2^K) at Romberg order K): the floating-point additions, multiplications and divisions the method
# performs on particle data as the oracle states it, tallied by the oracle's
# operation-counting build (oracle.op_counts on 8 particles x 1 turn; the counts
# do not depend on the particle), special functions listed apart and not
# charged.  tests/test_oracle_opcount.py recomputes these numbers.
ALGO_FLOPS_PER_PASS = {2: 671.4716, 3: 1239.8626, 4: 2338.9802}
ALGO_SPECIAL_PER_PASS = {2: {"sqrt": 20.4016, "sin_cos": 19.4029, "asin": 2.2827, "sinh_cosh": 7.9894},
                         3: {"sqrt": 38.0925, "sin_cos": 37.6645, "asin": 4.5654, "sinh_cosh": 15.9789},
                         4: {"sqrt": 72.9036, "sin_cos": 73.0462, "asin": 9.1308, "sinh_cosh": 31.9577}}
ALGO_FLOPS_PER_TYPE = {2: {"snake": 56.0, "quad_mk": 1645.0, "mult": 1053.0, "drift": 20.0, "sbend": 974.0}}
# The same count for the integrator comparison (Sec. 3.6, 5.3) on this ring:
# its drift-kick version (TEAPOT bends, drift-kick-drift quadrupoles) with two
# Romberg iterations and with the split-kick midpoint scheme, and the ring
# itself with the half-slice midpoint scheme and with two Romberg iterations.
ALGO_FLOPS_COMPARISON = {"drift_kick_romberg2": 601.8494, "drift_kick_mid_kick": 426.9379,
                         "bend_kick_mid_half": 678.0343, "bend_kick_romberg2": 671.4716}
# FP64 floating-point operations the FP64 tracker executes per particle-element
# pass on this workload (2 per DFMA, 1 per DADD/DMUL), and FP64-pipe
# instructions per pass, from the thread-level instruction counters of one ncu
# capture (profiles/track_fp64_rhic_like_ncu.md).  None until measured for the
# current kernel.
FP64_FLOPS_PER_PASS = 428.85
FP64_PIPE_INSTR_PER_PASS = 278.4
FP64_PIPE_LANES_PER_SM_CLOCK = 2
# DRAM bytes (read + write) per particle per launch of the FP64 tracker, from
# dram__bytes_read.sum + dram__bytes_write.sum of the same capture (2e4
# particles: 1.590 MB + 0 B), scaled linearly with the particle count.
FP64_DRAM_BYTES_PER_PARTICLE = 79.5


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--spin-order", type=int, default=2,
                    help="Romberg order 0..4, or -1 / -2 for the half-slice / split-kick midpoint schemes")
    ap.add_argument("--ring", choices=["rhic_like", "drift_kick"], default="rhic_like",
                    help="drift_kick: the same ring with TEAPOT bends and drift-kick-drift quadrupoles")
    ap.add_argument("--ggamma", type=float, default=45.5)
    ap.add_argument("--particles", type=int, default=None, help="override particles per GPU")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the mixed-precision variant report")
    ap.add_argument("--error-turns", type=int, default=1000, help="turns of the variants' error check")
    ap.add_argument("--profile-surrogate", type=int, default=0, metavar="TURNS",
                    help="run the learned map's turn loop for TURNS turns and exit (for ncu)")
    ap.add_argument("--profile-batch", type=int, default=0, metavar="TURNS",
                    help="track the 64-job batch TURNS turns, one launch per turn, and exit (for ncu)")
    ap.add_argument("--profile-train", type=int, default=0, metavar="STEPS",
                    help="profiling mode: only train the spin-map network for STEPS steps on 32768-row batches "
                         "(pairs from 4000 particles x 10 turns) and print the step time")
    return ap.parse_args()


def profile_train(args):
    """A short, self-contained run of the network's training kernels (for ncu)."""
    import torch
    import paper_1501_03450_b300 as st
    from paper_1501_03450_b300.surrogate import SpinMapSurrogate
    w = W.workload("rhic_like_spin_map", spin_order=args.spin_order)
    gg = w["ring"]["Ggamma0"]
    sg = SpinMapSurrogate(w["ring"], w["spin_order"], max_batch=w["batch"])
    z0, _ = W.gaussian_particles(4000, gg, seed=w["train_seed"], cut=w["cut"])
    pairs = sg.make_pairs_from_orbits(z0, 10)
    sg.fit_head(pairs, w["degree"])
    x, r = sg.targets(pairs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(sg.stream)
    sg.train(x, r, args.profile_train, batch=w["batch"], lr=w["lr"], log_every=0)
    e1.record(sg.stream)
    e1.synchronize()
    print(json.dumps({"profile_train_steps": args.profile_train, "batch": w["batch"],
                      "ms_per_step": e0.elapsed_time(e1) / max(1, args.profile_train),
                      "library": st.LIB_PATH}))
    sg.close()


def profile_surrogate(args):
    """A short run of the learned map's turn loop on the 10^4-particle
    averaging ensemble, with both orbit trackers (for ncu's launch list: the
    split of one turn into orbit, pack, network layers and spin step).  The
    network is untrained (its weights do not change the work)."""
    import torch
    import paper_1501_03450_b300 as st
    from paper_1501_03450_b300.surrogate import SpinMapSurrogate
    w = W.workload("rhic_like_spin_map", spin_order=args.spin_order)
    gg = w["ring"]["Ggamma0"]
    sg = SpinMapSurrogate(w["ring"], w["spin_order"], max_batch=w["n_particles"] + 128)
    z0, _ = W.gaussian_particles(2000, gg, seed=w["train_seed"], cut=w["cut"])
    pairs = sg.make_pairs_from_orbits(z0, 5)
    sg.fit_head(pairs, w["degree"])
    z, S = W.gaussian_particles(w["n_particles"], gg, seed=w["seed"] + 1, cut=w["cut"])
    out = {"profile_surrogate_turns": args.profile_surrogate, "particles": w["n_particles"], "library": st.LIB_PATH}
    for orbit in ("mixed", "fp64"):
        sg.track(z, S, 1, orbit=orbit)
        _, _, _, _, ms = sg.track(z, S, args.profile_surrogate, orbit=orbit)
        out[f"ms_per_turn_{orbit}_orbit"] = ms / max(1, args.profile_surrogate)
    print(json.dumps(out))
    sg.close()


def profile_batch(args):
    """One turn of the 64-job batch in one persistent launch (no graph), at
    --precision, in the default launch shape (for ncu: per-launch time and
    the spread of SM busy cycles, i.e. the tail of the work queue)."""
    import torch
    import paper_1501_03450_b300 as st
    jobs = W.batched_jobs(n_jobs=64, seed=20240603)
    b = st.Batch([W.with_spin_order(j["ring"], args.spin_order) for j in jobs], [j["n_particles"] for j in jobs],
                 args.precision)
    for k, j in enumerate(jobs):
        b.upload(k, *W.gaussian_particles(j["n_particles"], j["ring"]["Ggamma0"], seed=j["seed"]))
    b.set_launch(128, 1, 0, -1)
    for _ in range(args.profile_batch):
        b.track(1, args.spin_order)
    b.download(0)
    print(json.dumps({"profile_batch_turns": args.profile_batch, "precision": args.precision,
                      "library": st.LIB_PATH}))
    b.close()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu_index)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_rate(ring, z, S, spin_order, seconds_target=10.0, threads=None):
    """Time the FP64 oracle on a bounded sample of the workload on `threads`
    host threads (all cores by default); returns (passes/s, sample
    description, threads, particles)."""
    import oracle
    threads = threads or os.cpu_count() or 1
    n_el = len(ring["elements"])
    probe_n = min(z.shape[1], 4 * threads)
    t0 = time.perf_counter()
    oracle.track(ring, z[:, :probe_n], S[:, :probe_n], 1, spin_order, n_threads=threads)
    dt = max(time.perf_counter() - t0, 1e-6)
    rate = probe_n * n_el / dt
    n = int(min(z.shape[1], max(threads, rate * seconds_target / n_el)))
    t0 = time.perf_counter()
    oracle.track(ring, z[:, :n], S[:, :n], 1, spin_order, n_threads=threads)
    dt = time.perf_counter() - t0
    return n * n_el / dt, f"{n} particles x 1 turn of the {n_el}-element ring ({dt:.1f} s)", threads, n


def bench_config(args, npart, n_el, world):
    """The workload description both arms print (the GPU arm and the oracle
    reference arm time the same ring, ensemble, spin scheme and steps)."""
    K = args.spin_order
    return {"workload": f"{WORKLOAD}: 108-cell RHIC-like ring ({n_el} elements/turn)"
            + (", drift-kick version (TEAPOT bends, drift-kick-drift quadrupoles)" if args.ring == "drift_kick"
               else "")
            + f", {npart} Gaussian protons per GPU, Ggamma={args.ggamma}, "
            + (f"Romberg order {K}" if K >= 0 else ("half-slice" if K == -1 else "split-kick")
               + " midpoint spin scheme") + ", 1 turn per step",
            "ring": args.ring,
            "particles_per_gpu": npart, "elements_per_turn": n_el, "precision": args.precision,
            "spin_order": K, "turns_per_step": 1, "parallelism": f"replicas{world}",
            "l2": "GPU arm: flushed between steps (2x L2 buffer written outside the timed events)"}


def run_reference(args):
    rank, local_rank, world = dist_env()
    if rank != 0:
        return 0
    w = W.workload(WORKLOAD, spin_order=max(args.spin_order, 2) if args.spin_order < 0 else args.spin_order,
                   Ggamma0=args.ggamma)
    ring = w["ring"]
    if args.ring == "drift_kick":
        ring = W.drift_kick_ring(ring)
    n_el = len(ring["elements"])
    npart = args.particles or w["n_particles"]
    z, S = W.gaussian_particles(npart, args.ggamma, seed=w["seed"])
    import oracle
    threads = os.cpu_count() or 1
    # size each step for about 10 s of host work, so K + W steps stay within minutes
    _, _, _, n_step = oracle_rate(ring, z, S, args.spin_order, seconds_target=min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle.track(ring, z[:, :n_step], S[:, :n_step], 1, args.spin_order, n_threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.track(ring, z[:, :n_step], S[:, :n_step], 1, args.spin_order, n_threads=threads)
    dt = time.perf_counter() - t0
    value = n_step * n_el * args.steps / dt
    sample = f"{n_step} of {npart} particles x 1 turn per step ({n_el} elements)"
    out = {
        "impl": "reference", "metric": "particle-element passes/s", "value": value,
        "unit": "passes/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args, npart, n_el, args.gpus),
        "cpu_baseline": {"value": value, "unit": "passes/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "passes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


# ---------------------------------------------------------------------------
# variants: mixed precision (and the learned spin map) against the FP64 tracker
# ---------------------------------------------------------------------------

MIXED_WORKLOAD_PARTICLES = 1_000_000
FP64_MIDPOINT_PARTICLES = 100_000   # the FP64 tracker is fully occupied at 10^5
# FMA-pipe instructions the mixed tracker executes per pass on this workload
# (thread level: warp instructions x 32 / passes), from one ncu capture
# (profiles/track_mixed_rhic_like_ncu.md).  Packed FP32x2 instructions count
# once and the counters cannot tell them from scalar ones, so the executed
# measure is the share of the FMA pipe's issue slots (128 lanes per SM per
# clock), not a flop count.
MIXED_FMA_PIPE_INSTR_PER_PASS = 1344.0


def _tracker_rate(st, torch, ring, z, S, precision, spin_order, steps=3):
    """Passes/s of one tracker on a resident ensemble: CUDA events on the
    tracker's stream around single turns, L2 flushed between turns."""
    n = z.shape[1]
    stream = torch.cuda.Stream()
    lat = st.Lattice(ring)
    tr = st.Tracker(lat, n, precision, stream=stream.cuda_stream)
    tr.set_launch(block_threads=128, turns_per_launch=1)
    tr.upload(z, S)
    for _ in range(2):
        tr.track(1, spin_order)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            tr.track(1, spin_order)
            b.record(stream)
    torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in ev) * 1e-3
    tr.close()
    lat.close()
    return n * len(ring["elements"]) * steps / t


def variant_mixed(st, torch, args, fp64_value, fp32_peak):
    ring = W.with_spin_order(W.rhic_like_ring(args.ggamma), args.spin_order)
    n_el = len(ring["elements"])
    n = MIXED_WORKLOAD_PARTICLES
    z, S = W.gaussian_particles(n, args.ggamma, seed=3451)
    stream = torch.cuda.Stream()
    lat = st.Lattice(ring)
    tr = st.Tracker(lat, n, "mixed", stream=stream.cuda_stream)
    tr.set_launch(block_threads=128, turns_per_launch=1)
    tr.upload(z, S)
    for _ in range(2):
        tr.track(1, args.spin_order)
    torch.cuda.synchronize()
    steps = 3
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            tr.track(1, args.spin_order)
            b.record(stream)
    torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in ev) * 1e-3
    value = n * n_el * steps / t
    tr.close()
    lat.close()
    algo = ALGO_FLOPS_PER_PASS.get(args.spin_order)
    achieved = algo * n * n_el / (t / steps) / 1e12 if algo else None
    rate_now = n * n_el * steps / t
    sm_hz = 2032.0e6
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    fma_issue = MIXED_FMA_PIPE_INSTR_PER_PASS * rate_now / (128.0 * n_sm * sm_hz)
    out = {"metric": "particle-element passes/s", "value": value, "unit": "passes/s",
           "speedup_vs_fp64": value / fp64_value, "dtype": "f32 (compensated) + f64 per turn",
           "config": {"workload": f"108-cell RHIC-like ring, {n} Gaussian protons, Ggamma={args.ggamma}, "
                      f"Romberg order {args.spin_order}, 1 turn per step", "steps": steps},
           "roofline": {"bound": "alu", "pipe": "fp32", "achieved": achieved, "peak": fp32_peak / 1e12,
                        "unit": "TFLOP/s", "frac": achieved / (fp32_peak / 1e12) if achieved else None,
                        "algorithmic_flops_per_pass": algo,
                        "executed": {"fma_pipe_instr_per_pass": MIXED_FMA_PIPE_INSTR_PER_PASS,
                                     "fma_pipe_issue_frac_at_max_clock": fma_issue}},
           "error_vs_fp64": {}, "midpoint_schemes": {}}
    # the midpoint spin placements (Sec. 4.1) in both trackers, on the same ring
    # (order-2 slicing): mixed on the same 10^6 particles, FP64 on the headline 10^5
    ring_mid = W.with_spin_order(W.rhic_like_ring(args.ggamma), 2)
    for K, name in ((-1, "half_slice"), (-2, "split_kick")):
        r_mixed = _tracker_rate(st, torch, ring_mid, z, S, "mixed", K)
        r_fp64 = _tracker_rate(st, torch, ring_mid, z[:, :FP64_MIDPOINT_PARTICLES], S[:, :FP64_MIDPOINT_PARTICLES], "fp64", K)
        out["midpoint_schemes"][name] = {"spin_order": K, "mixed_passes_per_s": r_mixed,
                                         "fp64_passes_per_s": r_fp64, "speedup_vs_fp64": r_mixed / r_fp64}
    # accuracy: 1024-particle subset, mixed vs the FP64 tracker (pinned to the oracle)
    for gg in sorted({args.ggamma, 45.5, 487.0}):
        ring_g = W.with_spin_order(W.rhic_like_ring(gg), args.spin_order)
        zz, SS = W.gaussian_particles(1024, gg, seed=3451)
        zm, Sm, _ = st.track(ring_g, zz, SS, args.error_turns, args.spin_order, precision="mixed")
        zf, Sf, _ = st.track(ring_g, zz, SS, args.error_turns, args.spin_order, precision="fp64")
        dS = np.linalg.norm(Sm - Sf, axis=0)
        out["error_vs_fp64"][f"Ggamma={gg}"] = {
            "turns": args.error_turns, "particles": 1024, "dS_mean": float(dS.mean()), "dS_max": float(dS.max()),
            "orbit_max_abs": [float(x) for x in np.abs(zm - zf).max(axis=1)[:5]]}
    return out


def variant_batched(st, torch, args, turns=50):
    """64 uneven jobs (8-108 cells, G*gamma0 in [45.5, 487], 10^3-10^5
    particles) in one persistent launch per chunk of turns, replayed from a
    CUDA graph, in the launch shape the library's autotuner picks for each
    precision; CUDA events around `turns` of the configured 500 turns per job
    (every turn does the same work, so the rate is that of the whole 500).
    Against the same jobs tracked one after another on one stream with the
    single-job entry point (each job's turn timed with CUDA events, summed)."""
    jobs = W.batched_jobs(n_jobs=64, seed=20240603)
    for j in jobs:
        j["ring"] = W.with_spin_order(j["ring"], args.spin_order)
    passes_per_turn = sum(len(j["ring"]["elements"]) * j["n_particles"] for j in jobs)
    inputs = [W.gaussian_particles(j["n_particles"], j["ring"]["Ggamma0"], seed=j["seed"]) for j in jobs]
    out = {"config": {"workload": "64 seeded rings, 8-108 FODO cells, Ggamma U[45.5, 487], particles log-U[1e3, 1e5], "
                                  "500 turns per job configured",
                      "jobs": len(jobs), "particles": sum(j["n_particles"] for j in jobs),
                      "passes_per_turn": passes_per_turn, "turns_timed": turns,
                      "timing": "CUDA events on the batch stream around one graph replay of the timed turns"}}
    stream = torch.cuda.Stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) * 1e-3

    for prec in ("fp64", "mixed"):
        b = st.Batch([j["ring"] for j in jobs], [j["n_particles"] for j in jobs], prec, stream=stream.cuda_stream)
        for k in range(len(jobs)):
            b.upload(k, *inputs[k])
        tuned = b.autotune(args.spin_order, trial_turns=1)
        b.track(turns, args.spin_order)            # warm-up and graph capture
        torch.cuda.synchronize()
        dt = timed(lambda: b.track(turns, args.spin_order))
        b.close()
        # the same jobs one after another on one stream (single-job contexts),
        # one turn per job after a warm-up turn
        ds = 0.0
        for k, j in enumerate(jobs):
            lat = st.Lattice(j["ring"])
            tr = st.Tracker(lat, j["n_particles"], prec, stream=stream.cuda_stream)
            tr.set_launch(128, 1)
            tr.upload(*inputs[k])
            tr.track(1, args.spin_order)
            ds += timed(lambda: tr.track(1, args.spin_order))
            tr.close()
            lat.close()
        value = passes_per_turn * turns / dt
        out[prec] = {"value": value, "unit": "passes/s", "ms_per_turn": 1e3 * dt / turns,
                     "sequential_single_job_value": passes_per_turn / ds,
                     "speedup_vs_sequential": value / (passes_per_turn / ds), "autotuned_shape": tuned}
    return out


def variant_surrogate(st, torch, args, fp64_value, throughput_turns=30):
    """The learned one-turn spin map: trained here (pairs along tracked orbits,
    FP64 polynomial head, network on its own tensor-core kernels), then used
    for stroboscopic spin tracking with the orbit tracked exactly.  Error
    against plain FP64 spin tracking on 1024 particles after --error-turns
    turns (mean, percentiles, maximum).  Throughput on the 10^4-particle
    averaging ensemble and on 10^5 particles, each against the two trackers
    without the network on the same ensemble with the same stroboscopic sum:
    the mixed-precision tracker with its spin step (the fastest method without
    the network) and the FP64 tracker."""
    from paper_1501_03450_b300.surrogate import train_spin_map
    w = W.workload("rhic_like_spin_map", spin_order=args.spin_order)
    ring = w["ring"]
    gg = ring["Ggamma0"]
    n_el = len(ring["elements"])
    z_train, _ = W.gaussian_particles(w["train_particles"], gg, seed=w["train_seed"], cut=w["cut"])
    sg = train_spin_map(ring, z_train, w["train_turns"], w["spin_order"], degree=w["degree"], steps=w["steps"],
                        batch=w["batch"], lr=w["lr"], max_batch=100352)
    out = {"config": {"workload": f"108-cell RHIC-like ring, Ggamma={gg}, Romberg order {args.spin_order}; "
                      f"use: {w['n_particles']} Gaussian protons (cut {w['cut']} sigma), stroboscopic <S> at s=0",
                      "training": dict(sg.timings, degree=w["degree"], lr=w["lr"],
                                       pairs_from=f"{w['train_particles']} particles x {w['train_turns']} turns"),
                      "network": "6-256-256-256-256-4 SiLU, bf16 weights/activations, fp32 accumulation"}}
    # accuracy against plain FP64 tracking, orbit tracked in FP64 or by the
    # mixed tracker's compensated maps
    z, S = W.gaussian_particles(w["eval_particles"], gg, seed=w["seed"], cut=w["cut"])
    T = args.error_turns
    zp, Sp, _, avp, _ = sg.track_plain(z, S, T)
    out["error_vs_fp64"] = {}
    for orbit in ("fp64", "mixed"):
        zs, Ss, _, avs, _ = sg.track(z, S, T, orbit=orbit)
        dS = np.linalg.norm(Ss - Sp, axis=0)
        dA = np.linalg.norm(avs - avp, axis=0)
        p50, p90, p99 = np.percentile(dS, [50, 90, 99])
        out["error_vs_fp64"][f"orbit_{orbit}"] = {
            "turns": T, "particles": int(z.shape[1]), "dS_mean": float(dS.mean()), "dS_median": float(p50),
            "dS_p90": float(p90), "dS_p99": float(p99), "dS_max": float(dS.max()),
            "d_avgS_mean": float(dA.mean()), "d_avgS_max": float(dA.max()),
            "orbit_max_abs_diff": float(np.abs(zs[:4] - zp[:4]).max())}
    zm, Sm, _, avm, _ = sg.track_plain(z, S, T, precision="mixed")
    dm = np.linalg.norm(Sm - Sp, axis=0)
    out["error_vs_fp64"]["mixed_tracker"] = {"dS_mean": float(dm.mean()), "dS_max": float(dm.max()),
                                             "d_avgS_mean": float(np.linalg.norm(avm - avp, axis=0).mean())}
    p = sg.mlp.get_params()
    sg.mlp.set_params(np.zeros_like(p))
    _, Sl, _, _, _ = sg.track(z, S, T)
    sg.mlp.set_params(p)
    out["error_vs_fp64"]["polynomial_head_only_dS_mean"] = float(np.linalg.norm(Sl - Sp, axis=0).mean())
    # throughput: the averaging ensemble (10^4) and 10^5 particles, every
    # method with the stroboscopic sum, a bounded number of turns
    out["same_ensemble"] = {}
    for n in (w["n_particles"], 100000):
        zz, SS = W.gaussian_particles(n, gg, seed=w["seed"] + 1, cut=w["cut"])
        sg.track(zz, SS, 2, orbit="mixed")
        ms = {}
        _, _, _, _, ms["surrogate_mixed_orbit"] = sg.track(zz, SS, throughput_turns, orbit="mixed")
        _, _, _, _, ms["surrogate_fp64_orbit"] = sg.track(zz, SS, throughput_turns)
        _, _, _, _, ms["mixed_tracker"] = sg.track_plain(zz, SS, throughput_turns, precision="mixed")
        _, _, _, _, ms["fp64_tracker"] = sg.track_plain(zz, SS, throughput_turns)
        passes = n * n_el * throughput_turns
        rates = {k: passes / (v * 1e-3) for k, v in ms.items()}
        out["same_ensemble"][str(n)] = {
            "passes_per_s": rates, "ms_per_turn": {k: v / throughput_turns for k, v in ms.items()},
            "speedup_vs_mixed_same_ensemble": ms["mixed_tracker"] / ms["surrogate_mixed_orbit"],
            "speedup_vs_fp64_same_ensemble": ms["fp64_tracker"] / ms["surrogate_mixed_orbit"],
            "speedup_vs_fp64_same_ensemble_fp64_orbit": ms["fp64_tracker"] / ms["surrogate_fp64_orbit"]}
    head = out["same_ensemble"][str(w["n_particles"])]
    out.update({"metric": "particle-element passes/s", "value": head["passes_per_s"]["surrogate_mixed_orbit"],
                "unit": "passes/s", "orbit": "mixed (compensated FP32 maps)",
                "speedup_vs_mixed_same_ensemble": head["speedup_vs_mixed_same_ensemble"],
                "speedup_vs_plain_fp64_same_ensemble": head["speedup_vs_fp64_same_ensemble"],
                "speedup_vs_fp64_headline": head["passes_per_s"]["surrogate_mixed_orbit"] / fp64_value,
                "turns_timed": throughput_turns,
                "dtype": "f32 compensated orbit + bf16/fp32 network + f64 head and spin"})
    sg.close()
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def variant_fp64_configs(st, torch, npart, fp64_peak, seed):
    """FP64 pass rate on the RHIC-like ring at G gamma0 = 45.5 and 487 and
    Romberg orders 2, 3, 4 (slices max(4, 2^K)), one turn per launch, with the
    algorithmic roofline fraction of each."""
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    out = {}
    for gg in (45.5, 487.0):
        z, S = W.gaussian_particles(npart, gg, seed=seed)
        for K in (2, 3, 4):
            ring = W.workload(WORKLOAD, spin_order=K, Ggamma0=gg)["ring"]
            n_el = len(ring["elements"])
            lat = st.Lattice(ring)
            tr = st.Tracker(lat, npart, "fp64", stream=stream.cuda_stream)
            tr.set_launch(block_threads=128, turns_per_launch=1)
            tr.upload(z, S)
            tr.track(1, K)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
            with torch.cuda.stream(stream):
                for a, b in ev:
                    flush.zero_()
                    a.record(stream)
                    tr.track(1, K)
                    b.record(stream)
            torch.cuda.synchronize()
            t_s = sum(a.elapsed_time(b) for a, b in ev) * 1e-3 / len(ev)
            tr.close()
            lat.close()
            rate = npart * n_el / t_s
            algo = ALGO_FLOPS_PER_PASS.get(K)
            out[f"Ggamma={gg},K={K}"] = {"passes_per_s": rate, "ms_per_turn": 1e3 * t_s,
                                         "algorithmic_flops_per_pass": algo,
                                         "roofline_frac": algo * rate / fp64_peak if algo else None}
    return {"workload": f"108-cell RHIC-like ring, {npart} particles, 1 turn per launch", "configs": out}


def _time_turn(st, torch, ring, z, S, spin_order, flush, stream):
    """Seconds per turn of the FP64 tracker (one turn per launch, L2 flushed,
    mean of two launches after one warm-up)."""
    lat = st.Lattice(ring)
    tr = st.Tracker(lat, z.shape[1], "fp64", stream=stream.cuda_stream)
    tr.set_launch(block_threads=128, turns_per_launch=1)
    tr.upload(z, S)
    tr.track(1, spin_order)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            tr.track(1, spin_order)
            b.record(stream)
    torch.cuda.synchronize()
    tr.close()
    lat.close()
    return sum(a.elapsed_time(b) for a, b in ev) * 1e-3 / len(ev)


def variant_drift_kick(st, torch, npart, seed, fp64_peak, ggamma=45.5, dS_particles=4096):
    """The paper's comparison of integrators (Sec. 3.6, 5.3) on the RHIC-like
    ring: FP64 pass rates of the drift-kick version (TEAPOT bends,
    drift-kick-drift quadrupoles) with two Romberg iterations and with the
    split-kick midpoint scheme, of the bend-kick / matrix-kick ring with the
    half-slice midpoint scheme, and the one-turn mean spin error Delta S of
    each midpoint scheme without Romberg steps against bend-kick /
    matrix-kick tracking with 256 slices and three Romberg iterations (all
    tracked here on the GPU)."""
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    base = W.workload(WORKLOAD, spin_order=2, Ggamma0=ggamma)["ring"]
    dk = W.drift_kick_ring(base)
    n_el = len(base["elements"])
    z, S = W.gaussian_particles(npart, ggamma, seed=seed)
    rates = {}
    for name, ring, K in (("drift_kick_romberg2", dk, 2), ("drift_kick_mid_kick", dk, st.ST_SPIN_MID_KICK),
                          ("bend_kick_mid_half", base, st.ST_SPIN_MID_HALF), ("bend_kick_romberg2", base, 2)):
        rates[name] = npart * n_el / _time_turn(st, torch, ring, z, S, K, flush, stream)
    zs, Ss = W.gaussian_particles(dS_particles, ggamma, seed=seed + 1)
    _, Sref, _ = st.track(W.with_slices(base, 256), zs, Ss, 1, 3)
    dS = {}
    for nb in (4, 16, 64):
        row = {}
        for name, ring, K in (("drift_kick_mid_kick", dk, st.ST_SPIN_MID_KICK),
                              ("drift_kick_mid_half", dk, st.ST_SPIN_MID_HALF),
                              ("bend_kick_mid_half", base, st.ST_SPIN_MID_HALF)):
            _, S1, _ = st.track(W.with_slices(ring, nb), zs, Ss, 1, K)
            row[name] = float(np.linalg.norm(S1 - Sref, axis=0).mean())
        row["drift_kick_over_bend_kick"] = row["drift_kick_mid_kick"] / row["bend_kick_mid_half"]
        dS[f"n_b={nb}"] = row
    roof = {k: {"algorithmic_flops_per_pass": ALGO_FLOPS_COMPARISON[k],
                "frac_of_fp64_peak": ALGO_FLOPS_COMPARISON[k] * v / fp64_peak} for k, v in rates.items()}
    # the drift-kick ring in the mixed-precision tracker (TEAPOT bends in compensated
    # FP32), on the mixed tracker's 10^6-particle ensemble
    zm, Sm = W.gaussian_particles(MIXED_WORKLOAD_PARTICLES, ggamma, seed=seed)
    mixed = {}
    for name, K in (("drift_kick_romberg2", 2), ("drift_kick_mid_kick", st.ST_SPIN_MID_KICK)):
        r = _tracker_rate(st, torch, dk, zm, Sm, "mixed", K)
        mixed[name] = {"passes_per_s": r, "speedup_vs_fp64": r / rates[name]}
    return {"workload": f"108-cell RHIC-like ring at G gamma0 = {ggamma}, {npart} particles, 1 turn per launch",
            "passes_per_s": rates, "roofline": roof, "one_turn_dS": dS,
            "mixed": dict(mixed, particles=MIXED_WORKLOAD_PARTICLES),
            "dS_sample": f"{dS_particles} particles, reference: bend-kick/matrix-kick, 256 slices, 3 Romberg "
                         "iterations"}


def element_type_breakdown(st, torch, ring, npart, seed, K, ggamma, min_elements=200, precision="fp64"):
    """Pass rate of the tracker (FP64 or mixed) per element type: for each type in the
    ring, a ring made of that type's elements only (in ring order, repeated
    to at least min_elements) is tracked for one turn on the same ensemble
    size; its share of the full ring's time is count / rate normalised."""
    z, S = W.gaussian_particles(npart, ggamma, seed=seed)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    out = {}
    for t in dict.fromkeys(e["type"] for e in ring["elements"]):
        els = [e for e in ring["elements"] if e["type"] == t]
        reps = -(-min_elements // len(els))
        sub = dict(ring, elements=els * reps, name=f"{t}_only")
        lat = st.Lattice(sub)
        tr = st.Tracker(lat, npart, precision, stream=stream.cuda_stream)
        tr.set_launch(block_threads=128, turns_per_launch=1)
        tr.upload(z, S)
        tr.track(1, K)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
        with torch.cuda.stream(stream):
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                tr.track(1, K)
                b.record(stream)
        torch.cuda.synchronize()
        t_s = sum(a.elapsed_time(b) for a, b in ev) * 1e-3 / len(ev)
        tr.close()
        lat.close()
        rate = npart * len(sub["elements"]) / t_s
        algo = ALGO_FLOPS_PER_TYPE.get(K, {}).get(t)
        out[t] = {"passes_per_s": rate, "count_in_ring": len(els), "slices": sorted({e["n_slices"] for e in els}),
                  "algorithmic_flops_per_pass": algo, "algorithmic_tflops": algo * rate / 1e12 if algo else None}
    total = sum(v["count_in_ring"] / v["passes_per_s"] for v in out.values())
    for v in out.values():
        v["time_share"] = v["count_in_ring"] / v["passes_per_s"] / total
    return {"workload": f"one element type per ring, {npart} particles, {precision}, order {K}, 1 turn",
            "types": out, "predicted_ring_passes_per_s": len(ring["elements"]) / total}


def main():
    args = parse_args()
    if args.profile_train:
        return profile_train(args)
    if args.profile_surrogate:
        return profile_surrogate(args)
    if args.profile_batch:
        return profile_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_1501_03450_b300 as st
    from paper_1501_03450_b300.replicas import aggregate_rate, max_over_ranks, rank_seed

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    # the midpoint schemes run on the slicing of Romberg order 2 (4 slices per
    # element), the ring of the integrator comparison
    w = W.workload(WORKLOAD, spin_order=max(args.spin_order, 2) if args.spin_order < 0 else args.spin_order,
                   Ggamma0=args.ggamma)
    ring = w["ring"]
    if args.ring == "drift_kick":
        ring = W.drift_kick_ring(ring)
    n_el = len(ring["elements"])
    npart = args.particles or w["n_particles"]
    z, S = W.gaussian_particles(npart, args.ggamma, seed=rank_seed(w["seed"], rank))
    K = args.spin_order
    headline = args.ring == "rhic_like" and K >= 0

    stream = torch.cuda.Stream()
    lat = st.Lattice(ring)
    tr = st.Tracker(lat, npart, args.precision, stream=stream.cuda_stream)
    tr.set_launch(block_threads=128, turns_per_launch=1)
    tr.upload(z, S)
    fp64_peak, fp32_peak = st.st_measure_peaks()
    fp32x2_peak = st.st_measure_fp32x2_peak()

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    launches_per_step = 1

    # warm-up
    for _ in range(args.warmup):
        tr.track(1, K)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[local_rank]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").replace(",", "").isdigit() else local_rank
    sampler = ClockSampler(gpu_index)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()                      # evict L2 between steps (outside the timed events)
            starts[i].record(stream)
            tr.track(1, K)
            ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_sum = max_over_ranks(sum(step_ms) * 1e-3, dist, "cuda")
    passes_per_rank = npart * n_el * args.steps
    value = aggregate_rate(passes_per_rank, world, t_sum)

    # ---- end to end through the C ABI with host buffers -------------------
    e2e = None
    if not args.no_e2e:
        zh = torch.from_numpy(z).pin_memory()
        Sh = torch.from_numpy(S).pin_memory()
        zo = torch.empty_like(zh).pin_memory()
        So = torch.empty_like(Sh).pin_memory()
        lo = torch.empty(npart, dtype=torch.uint8).pin_memory()
        e2e_steps = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            st.st_particles_upload(tr.handle, zh.data_ptr(), Sh.data_ptr(), 0)
            tr.track(1, K)
            st.st_spins_download(tr.handle, So.data_ptr(), zo.data_ptr(), lo.data_ptr(), 0)
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": aggregate_rate(npart * n_el * e2e_steps, world, te), "unit": "passes/s",
               "h2d_bytes_per_step": 9 * 8 * npart, "d2h_bytes_per_step": 9 * 8 * npart + npart}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the tracking kernel ---------------------------------
    peak = fp64_peak if args.precision == "fp64" else fp32_peak
    avg_launch_s = t_sum / (args.steps * launches_per_step)
    passes_per_launch = npart * n_el
    if headline:
        algo = ALGO_FLOPS_PER_PASS.get(K)
    else:
        algo = {("drift_kick", 2): ALGO_FLOPS_COMPARISON["drift_kick_romberg2"],
                ("drift_kick", -2): ALGO_FLOPS_COMPARISON["drift_kick_mid_kick"],
                ("rhic_like", -1): ALGO_FLOPS_COMPARISON["bend_kick_mid_half"]}.get((args.ring, K))
    achieved = algo * passes_per_launch / avg_launch_s / 1e12 if algo else None
    executed = None
    if args.precision == "fp64" and K == 2 and headline and FP64_FLOPS_PER_PASS:
        ex_tflops = FP64_FLOPS_PER_PASS * passes_per_launch / avg_launch_s / 1e12
        issue = FP64_PIPE_INSTR_PER_PASS * passes_per_launch / avg_launch_s
        sm_hz = (clocks.get("sm_mhz") or 2032.0) * 1e6
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
        executed = {"fp64_flops_per_pass": FP64_FLOPS_PER_PASS, "tflops": ex_tflops,
                    "frac_of_peak": ex_tflops / (peak / 1e12),
                    "fp64_pipe_instr_per_pass": FP64_PIPE_INSTR_PER_PASS,
                    "pipe_issue_frac": issue / (FP64_PIPE_LANES_PER_SM_CLOCK * n_sm * sm_hz)}
    roofline = {"bound": "alu", "pipe": "fp64" if args.precision == "fp64" else "fp32",
                "achieved": achieved, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": (achieved / (peak / 1e12)) if achieved else None,
                "traffic": FP64_DRAM_BYTES_PER_PARTICLE * npart if args.precision == "fp64" and headline else None,
                "peak_source": "measured by st_measure_peaks (independent FMA chains) at run time",
                "algorithmic_flops_per_pass": algo,
                "algorithmic_basis": "additions, multiplications and divisions on particle data counted by the "
                                     "oracle's operation-counting build for this ring and order; special functions "
                                     "per pass not charged: " + json.dumps(ALGO_SPECIAL_PER_PASS.get(K) if headline
                                                                           else None),
                "executed": executed}

    breakdown = None
    if not args.no_variants and world == 1 and args.precision == "fp64":
        breakdown = element_type_breakdown(st, torch, ring, npart, w["seed"], K, args.ggamma)

    variants = None
    if not args.no_variants and world == 1:
        variants = {"fp64_configs": variant_fp64_configs(st, torch, npart, fp64_peak, w["seed"]),
                    "drift_kick": variant_drift_kick(st, torch, npart, w["seed"], fp64_peak),
                    "mixed": variant_mixed(st, torch, args, value, fp32_peak),
                    "batched": variant_batched(st, torch, args),
                    "surrogate": variant_surrogate(st, torch, args, value)}

    cpu = None
    if not args.no_cpu_baseline:
        rate, sample, threads, _ = oracle_rate(ring, z, S, K)
        rate1, sample1, _, _ = oracle_rate(ring, z, S, K, seconds_target=3.0, threads=1)
        cpu = {"value": rate, "unit": "passes/s", "cores": threads, "kind": "oracle", "sample": sample,
               "value_1_core": rate1, "sample_1_core": sample1}

    out = {
        "metric": "particle-element passes/s", "value": value, "unit": "passes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_sum / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": bench_config(args, npart, n_el, world),
        "e2e": e2e,
        "gpu_launches": args.steps * launches_per_step,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "per_element_type": breakdown,
        "variants": variants,
        "clocks": clocks,
        "wall_s_timed": wall,
        "peaks_measured": {"fp64_tflops": fp64_peak / 1e12, "fp32_tflops": fp32_peak / 1e12,
                           "fp32x2_tflops": fp32x2_peak / 1e12},
    }
    print(json.dumps(out))
    tr.close()
    lat.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
