"""The operation-counting build of the oracle (the roofline's algorithmic
work per pass): it counts what the oracle's formulas state, it computes the
same numbers as the oracle, counts scale with particles and turns, and the
bench's per-pass figures are what it counts today."""
import importlib.util
import os

import numpy as np

import oracle
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_consts", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_drift_pass_counts_the_drift_formula():
    """Eq. (29b) as written: P^2 = 1 + 2 Pt/beta0 + Pt^2 (2 add, 2 mul, 1 div),
    Ps^2 = P^2 - Px^2 - Py^2 (2 add, 2 mul), Ps (1 sqrt), X and Y (1 mul,
    1 div, 1 add each), T += s (1/beta0 - (1/beta0 + Pt)/Ps) (3 add, 1 mul,
    1 div; 1/beta0 is a constant)."""
    ring = W.single_element_ring(W.element("drift", L=2.0), 45.5)
    z, S = W.gaussian_particles(5, 45.5, seed=1)
    c, _, _, _ = oracle.op_counts(ring, z, S, 1, 0)
    assert {k: v / 5 for k, v in c.items()} == dict(add=9, mul=7, div=4, sqrt=1, sincos=0, tan=0, asin=0,
                                                    sinh_cosh=0)


def test_counting_build_computes_what_the_oracle_computes():
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    z, S = W.gaussian_particles(16, 45.5, seed=2)
    _, zc, Sc, lc = oracle.op_counts(ring, z, S, 3, 2)
    zo, So, lo = oracle.track(ring, z, S, 3, 2)
    assert np.array_equal(lc, lo)
    assert np.abs(zc - zo).max() < 1e-15 and np.abs(Sc - So).max() < 1e-15


def test_counts_scale_with_particles_and_turns():
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    z, S = W.gaussian_particles(12, 45.5, seed=3)
    c1, _, _, _ = oracle.op_counts(ring, z[:, :6], S[:, :6], 1, 2)
    c2, _, _, _ = oracle.op_counts(ring, z, S, 1, 2)
    c3, _, _, _ = oracle.op_counts(ring, z[:, :6], S[:, :6], 2, 2)
    assert all(c2[k] == 2 * c1[k] == c3[k] for k in c1)


def test_bench_algorithmic_figures_are_current():
    b = _bench()
    w = W.workload("rhic_like_1e5")
    ring = w["ring"]
    z, S = W.gaussian_particles(8, 45.5, seed=1)
    c, _, _, _ = oracle.op_counts(ring, z, S, 1, 2)
    passes = 8 * len(ring["elements"])
    assert abs((c["add"] + c["mul"] + c["div"]) / passes - b.ALGO_FLOPS_PER_PASS[2]) < 1e-3
    sp = b.ALGO_SPECIAL_PER_PASS[2]
    assert abs(c["sqrt"] / passes - sp["sqrt"]) < 1e-3 and abs(c["sincos"] / passes - sp["sin_cos"]) < 1e-3
    assert abs(c["asin"] / passes - sp["asin"]) < 1e-3 and abs(c["sinh_cosh"] / passes - sp["sinh_cosh"]) < 1e-3
    for K in (3, 4):
        rk = W.workload("rhic_like_1e5", spin_order=K)["ring"]
        ck, _, _, _ = oracle.op_counts(rk, z, S, 1, K)
        assert abs((ck["add"] + ck["mul"] + ck["div"]) / (8 * len(rk["elements"])) - b.ALGO_FLOPS_PER_PASS[K]) < 1e-3
    for t, v in b.ALGO_FLOPS_PER_TYPE[2].items():
        els = [e for e in ring["elements"] if e["type"] == t]
        ct, _, _, _ = oracle.op_counts(dict(ring, elements=els), z, S, 1, 2)
        assert (ct["add"] + ct["mul"] + ct["div"]) / (8 * len(els)) == v


def test_bench_comparison_figures_are_current():
    """Algorithmic work per pass of the integrator comparison (drift-kick ring
    with Romberg and split-kick midpoint schemes; the ring with the
    half-slice midpoint scheme and with Romberg)."""
    b = _bench()
    base = W.workload("rhic_like_1e5")["ring"]
    dk = W.drift_kick_ring(base)
    z, S = W.gaussian_particles(8, 45.5, seed=1)
    for name, ring, K in (("drift_kick_romberg2", dk, 2), ("drift_kick_mid_kick", dk, oracle.MID_KICK),
                          ("bend_kick_mid_half", base, oracle.MID_HALF), ("bend_kick_romberg2", base, 2)):
        c, _, _, _ = oracle.op_counts(ring, z, S, 1, K)
        per_pass = (c["add"] + c["mul"] + c["div"]) / (8 * len(ring["elements"]))
        assert abs(per_pass - b.ALGO_FLOPS_COMPARISON[name]) < 1e-3, name
