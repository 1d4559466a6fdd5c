"""Learned one-turn spin map: training pairs from the FP64 tracker, training
by the network's own tensor-core kernels, and stroboscopic spin tracking with
the map while the orbit is tracked exactly.

The map sends a particle's orbit z = (X, Px, Y, Py, T, Pt) at the start of the
lattice (the fixed azimuth s = 0) to the unit quaternion of its spin rotation
over one turn (the composed element rotations of Sec. 4, Eqs. (37)-(39)):

    q(z) = normalise(q0 + P(x) + s y(x)),   x = in_scale * z,

q0 the one-turn quaternion of the on-axis particle, P a polynomial (degree
<= 3) fitted by FP64 least squares on the tracked pairs, y the 6 -> 256 x 4 ->
4 SiLU network (bf16 weights and activations, FP32 accumulation) trained on
the residual (q - q0 - P(x)) / s, and s the residual's RMS.  T enters with
scale 0: no element of these rings depends on the arrival time (no RF), so the
one-turn map does not depend on T.

Every per-sample step runs in the CUDA library (pair tracking, the fit's
moments, the residual targets, forward, backward, Adam, the surrogate turn
loop).  The host does the bookkeeping: the initial weights, the batch and
learning-rate schedule.  PyTorch provides device memory and the stream.
"""
from __future__ import annotations

import math
from typing import Dict, Optional

import numpy as np
import torch

from . import MLP, Lattice, Tracker, st_track_average, st_track_one_turn_map, st_track_surrogate

LAYERS = [(256, 6), (256, 256), (256, 256), (256, 256), (4, 256)]


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def init_params(seed: int, gain: float = 1.0, last_scale: float = 0.1) -> np.ndarray:
    """Initial network weights, flattened W1, b1, ..., W5, b5: normal with std
    gain * sqrt(2 / fan_in) (the output layer scaled by last_scale), biases 0."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (r, c) in enumerate(LAYERS):
        std = gain * math.sqrt(2.0 / c) * (last_scale if l == len(LAYERS) - 1 else 1.0)
        parts.append(rng.standard_normal(r * c) * std)
        parts.append(np.zeros(r))
    return np.concatenate(parts)


class SpinMapSurrogate:
    """Learned one-turn spin map of one ring at one reference energy."""

    def __init__(self, ring: Dict, spin_order: int = 2, max_batch: int = 65536, seed: int = 1501):
        if not torch.cuda.is_available():
            raise RuntimeError("SpinMapSurrogate needs a CUDA device")
        self.ring = ring
        self.spin_order = int(spin_order)
        self.stream = torch.cuda.Stream()
        self.sp = self.stream.cuda_stream
        self.lattice = Lattice(ring)
        self.max_batch = int(max_batch)
        self.mlp = MLP(self.max_batch, self.sp)
        self.seed = int(seed)
        self.q0 = self.closed_orbit_quaternion()
        self.in_scale = None
        self.coef = None
        self.degree = None
        self.out_scale = np.ones(4)
        self.history = []

    # ---------------------------------------------------------------- tracking
    def _tracker(self, n: int) -> Tracker:
        return Tracker(self.lattice, n, "fp64", self.sp)

    def one_turn_maps(self, z: np.ndarray, q_ref) -> np.ndarray:
        """One-turn quaternions [4, n] of the orbits z [6, n] (host)."""
        n = z.shape[1]
        tr = self._tracker(n)
        try:
            S = np.zeros((3, n))
            S[1] = 1.0
            tr.upload(z, S)
            with torch.cuda.stream(self.stream):
                q = torch.empty((4, n), dtype=torch.float64, device="cuda")
            st_track_one_turn_map(tr.handle, self.spin_order, q_ref, _ptr(q))
            self.stream.synchronize()
            return q.cpu().numpy()
        finally:
            tr.close()

    def closed_orbit_quaternion(self) -> np.ndarray:
        """q0: the one-turn quaternion of the on-axis particle (scalar part >= 0)."""
        return self.one_turn_maps(np.zeros((6, 1)), [1.0, 0.0, 0.0, 0.0])[:, 0].copy()

    # ------------------------------------------------------------ training set
    def make_pairs_from_orbits(self, z0: np.ndarray, n_turns: int, S0: Optional[np.ndarray] = None):
        """Pairs along tracked orbits: the ensemble z0 [6, m] is tracked for
        n_turns (FP64) and every turn contributes (z at s = 0, one-turn
        quaternion) for every particle, so that the pairs sample the region
        of phase space the orbits of such an ensemble visit.  Pairs are
        ordered turn by turn; m * n_turns in all."""
        m = z0.shape[1]
        n = m * int(n_turns)
        tr = self._tracker(m)
        try:
            with torch.cuda.stream(self.stream):
                z64 = torch.empty((6, n), dtype=torch.float64, device="cuda")
                q64 = torch.empty((4, n), dtype=torch.float64, device="cuda")
                zt = torch.empty((6, m), dtype=torch.float64, device="cuda")
                qt = torch.empty((4, m), dtype=torch.float64, device="cuda")
                st_ = torch.empty((3, m), dtype=torch.float64, device="cuda")
                lost = torch.empty(m, dtype=torch.uint8, device="cuda")
            S = np.zeros((3, m))
            S[1] = 1.0
            tr.upload(z0, S if S0 is None else S0)
            for t in range(int(n_turns)):
                tr.download_device(_ptr(st_), _ptr(zt), None)
                st_track_one_turn_map(tr.handle, self.spin_order, self.q0, _ptr(qt))
                with torch.cuda.stream(self.stream):
                    z64[:, t * m:(t + 1) * m].copy_(zt)
                    q64[:, t * m:(t + 1) * m].copy_(qt)
            tr.download_device(_ptr(st_), None, _ptr(lost))
            self.stream.synchronize()
        finally:
            tr.close()
        n_lost = int(lost.cpu().numpy().sum())
        if n_lost:
            raise RuntimeError(f"make_pairs_from_orbits: {n_lost} orbits were lost")
        return dict(z=z64.cpu().numpy(), z64=z64, q64=q64, lost=torch.zeros(n, dtype=torch.uint8, device="cuda"),
                    n=n)

    def fit_head(self, pairs: Dict, degree: int = 3, in_scale=None):
        """Input scales (1 / RMS of each coordinate over the pairs; 0 for T),
        the FP64 least-squares polynomial P of the given degree, and the output
        scales s_k = RMS of each component of the residual q - q0 - P(x), so
        that the network's targets are O(1) in every component."""
        if in_scale is None:
            rms = np.sqrt(np.mean(pairs["z"] ** 2, axis=1))
            in_scale = np.where(rms > 0, 1.0 / np.where(rms > 0, rms, 1.0), 0.0)
            in_scale[4] = 0.0
        self.in_scale = np.asarray(in_scale, dtype=np.float64)
        self.degree = int(degree)
        self.mlp.set_head(self.q0, None, 1.0, self.in_scale)
        self.coef, self.fit_rms = self.mlp.fit_head(self.degree, _ptr(pairs["z64"]), _ptr(pairs["q64"]),
                                                    pairs["n"], _ptr(pairs["lost"]))
        self.out_scale = np.where(self.fit_rms > 0, self.fit_rms, 1.0)
        self.mlp.set_scale(self.out_scale)
        return self.in_scale, self.coef, self.out_scale

    def targets(self, pairs: Dict):
        """The network's training rows for the pairs with the current head:
        x [n, 6] (float orbit) and r [n, 4] = (q - q0 - P(x)) / s."""
        n = pairs["n"]
        with torch.cuda.stream(self.stream):
            x = torch.empty((n, 6), dtype=torch.float32, device="cuda")
            r = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        self.mlp.make_targets(_ptr(pairs["z64"]), _ptr(pairs["q64"]), n, _ptr(x), _ptr(r))
        self.stream.synchronize()
        return x, r

    def train(self, x: torch.Tensor, r: torch.Tensor, steps: int, batch: int = 16384, lr: float = 1e-3,
              lr_final: float = 1e-6, log_every: int = 500, init_seed: int = None, warmup: int = 200):
        """Adam on the residual regression mean |y - r|^2 over contiguous
        batches of the (randomly ordered) rows; the learning rate warms up
        linearly and then decays as a cosine from lr to lr_final.  The
        schedule (each step's first row and learning rate) is computed here
        and the steps run in one library call."""
        n = x.shape[0]
        batch = min(int(batch), self.max_batch, n)
        self.mlp.set_params(init_params(self.seed if init_seed is None else init_seed))
        rng = np.random.default_rng(self.seed + 1)
        start = int(rng.integers(0, n - batch + 1))
        starts = np.empty(steps, dtype=np.int64)
        lrs = np.empty(steps, dtype=np.float32)
        for k in range(steps):
            if start + batch > n:
                start = int(rng.integers(0, batch)) if n >= 2 * batch else 0
            starts[k] = start
            start += batch
            f = min(1.0, (k + 1) / warmup) if warmup else 1.0
            c = 0.5 * (1 + math.cos(math.pi * k / max(1, steps - 1)))
            lrs[k] = f * (lr_final + (lr - lr_final) * c)
        losses = self.mlp.train(_ptr(x), _ptr(r), n, batch, starts, lrs, want_loss=bool(log_every))
        if log_every:
            for k in range(steps):
                if k % log_every == 0 or k == steps - 1:
                    self.history.append((k, float(losses[k])))
        return self.history

    def eval_loss(self, x: torch.Tensor, r: torch.Tensor) -> float:
        """Mean |y - r|^2 of the current network over the given rows."""
        n = x.shape[0]
        tot, k = 0.0, 0
        while k < n:
            b = min(self.max_batch, n - k)
            loss, _ = self.mlp.loss_grad_residual(_ptr(x) + k * 24, _ptr(r) + k * 16, b)
            tot += loss * b
            k += b
        return tot / n

    # ------------------------------------------------------------------- use
    def track(self, z: np.ndarray, S: np.ndarray, n_turns: int, average: bool = True, timed: bool = False,
              orbit: str = "fp64"):
        """Stroboscopic tracking with the learned map: returns (z, S, lost,
        <S> or None, ms).  orbit: "fp64" or "mixed" (the mixed tracker's
        compensated orbit maps)."""
        return _run(self, z, S, n_turns, average, timed, surrogate=True, orbit=orbit)

    def track_plain(self, z: np.ndarray, S: np.ndarray, n_turns: int, average: bool = True,
                    timed: bool = False, precision: str = "fp64"):
        """The same with plain spin tracking: precision "fp64" (the reference
        for the map's error) or "mixed" (the mixed-precision tracker with its
        spin step, the fastest method without the network)."""
        return _run(self, z, S, n_turns, average, timed, surrogate=False, orbit=precision)

    def close(self):
        self.mlp.close()
        self.lattice.close()


def _run(sg: SpinMapSurrogate, z, S, n_turns, average, timed, surrogate, orbit="fp64"):
    n = z.shape[1]
    if surrogate and n > sg.max_batch:
        raise ValueError("more particles than the network's max_batch")
    tr = Tracker(sg.lattice, n, orbit, sg.sp)
    try:
        with torch.cuda.stream(sg.stream):
            ssum = torch.zeros((3, n), dtype=torch.float64, device="cuda") if average else None
        tr.upload(z, S)
        sg.stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sg.stream)
        if surrogate:
            st_track_surrogate(tr.handle, sg.mlp.handle, n_turns, _ptr(ssum) if average else None)
        elif average:
            st_track_average(tr.handle, n_turns, sg.spin_order, _ptr(ssum))
        else:
            tr.track(n_turns, sg.spin_order)
        e1.record(sg.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        z1, S1, lost = tr.download()
        avg = (ssum.cpu().numpy() / max(1, n_turns)) if average else None
        return z1, S1, lost, avg, ms
    finally:
        tr.close()


def train_spin_map(ring: Dict, z_train: np.ndarray, sample_turns: int, spin_order: int = 2, degree: int = 3,
                   steps: int = 20000, batch: int = 32768, lr: float = 1e-3, seed: int = 1501,
                   max_batch: int = 65536) -> SpinMapSurrogate:
    """The whole training recipe: pairs along the orbits of the ensemble
    z_train [6, m] over sample_turns turns (m * sample_turns pairs), the FP64
    polynomial head of the given degree, and `steps` Adam steps of the
    network on the residual.  Returns the trained surrogate; its `timings`
    holds the seconds spent on pairs, fit and training."""
    import time
    sg = SpinMapSurrogate(ring, spin_order, max_batch=max_batch, seed=seed)
    t0 = time.perf_counter()
    pairs = sg.make_pairs_from_orbits(z_train, sample_turns)
    t1 = time.perf_counter()
    sg.fit_head(pairs, degree)
    x, r = sg.targets(pairs)
    t2 = time.perf_counter()
    sg.train(x, r, steps, batch=batch, lr=lr)
    t3 = time.perf_counter()
    sg.timings = dict(pairs_s=t1 - t0, fit_s=t2 - t1, train_s=t3 - t2, n_pairs=pairs["n"], steps=steps,
                      batch=min(batch, max_batch, pairs["n"]))
    del pairs, x, r
    return sg
