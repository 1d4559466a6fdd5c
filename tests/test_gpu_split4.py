"""GPU parity of the fourth-order slice maps (Sec. 3.3: Yoshida's composition
of the symmetric drift-kick and matrix-kick maps of Eq. (27)): the CUDA FP64
tracker through the C ABI against the CPU oracle at 1e-11 for single
elements at every Romberg order, a RHIC-like ring with fourth-order maps and
fringe kicks, and the batched entry point; the CUDA result's own rate of
convergence to the Thomas-BMT ODE through a strong multipole; and the
mixed-precision tracker's fourth-order slices within its error budget."""
import math
import os
import sys

import numpy as np
import pytest

import oracle
import paper_1501_03450_b300 as st
import workloads as W

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from ode_reference import integrate  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-11


def compare(ring, z, S, turns, K, tol=TOL):
    zg, Sg, lg = st.track(ring, z, S, turns, K)
    zo, So, lo = oracle.track(ring, z, S, turns, K)
    assert np.array_equal(lg, lo)
    dz = np.abs(zg - zo).max(axis=1)
    ds = np.abs(Sg - So).max()
    assert dz.max() < tol and ds < tol, (dz, ds)
    return zg, Sg, lg


ELEMENTS = [
    W.element("mult", L=1.0, n_slices=8, k1=0.3, k2=5.0, split_order=4),
    W.element("quad_mk", L=1.0, n_slices=8, k1=0.3, split_order=4),
    W.element("quad_mk", L=1.0, n_slices=8, k1=-0.3, split_order=4),
]


@pytest.mark.parametrize("el", ELEMENTS, ids=["dkd", "mk_f", "mk_d"])
@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_single_fourth_order_element_every_order(el, K):
    gg = 45.5
    ring = W.single_element_ring(el, gg)
    z, S = W.gaussian_particles(257, gg, seed=90 + K, sigmas=dict(x=3e-3, y=3e-3))
    compare(ring, z, S, 10, K)


def test_rhic_like_ring_fourth_order_with_fringes():
    ring = W.with_fringes(W.with_split_order(W.with_spin_order(W.rhic_like_ring(45.5, n_cells=20), 2), 4))
    z, S = W.gaussian_particles(300, 45.5, seed=31)
    compare(ring, z, S, 10, 2)


def test_batched_jobs_fourth_order():
    rings = [W.with_split_order(W.with_spin_order(W.rhic_like_ring(gg, n_cells=c), 2), 4)
             for gg, c in ((45.5, 6), (300.0, 8))]
    rings.append(W.with_spin_order(W.toy_ring(45.5), 2))
    ns = [150, 97, 64]
    b = st.Batch(rings, ns, "fp64")
    inputs = []
    for k, (ring, n) in enumerate(zip(rings, ns)):
        z, S = W.gaussian_particles(n, ring["Ggamma0"], seed=95 + k)
        b.upload(k, z, S)
        inputs.append((z, S))
    b.track(3, 2)
    for k, (ring, (z, S)) in enumerate(zip(rings, inputs)):
        zb, Sb, lb = b.download(k)
        zo, So, lo = oracle.track(ring, z, S, 3, 2)
        assert np.array_equal(lb, lo)
        assert np.abs(zb - zo).max() < TOL and np.abs(Sb - So).max() < TOL
    b.close()


def test_cuda_spin_converges_at_the_orbit_order():
    """Strong drift-kick multipole, one Romberg iteration, tracked by the
    CUDA tracker: the spin error against the Thomas-BMT ODE falls as N^-4
    with the fourth-order map and as N^-2 with the second-order one."""
    gg = 45.5
    G = W.G_PROTON
    z0 = np.array([3e-3, 3e-4, -2e-3, 2e-4, 0.0, float(W.delta_to_pt(np.array(2e-3), gg))])
    S0 = np.array([0.3, 0.2, math.sqrt(1 - 0.13)])
    _, Sref = integrate("mult", z0, 1.0, G, gg, k1=0.5, k2=5.0, S0=S0)
    for order, lo, hi in ((4, 14.0, 18.0), (2, 3.6, 4.4)):
        e = []
        for N in (4, 8, 16, 32):
            ring = W.single_element_ring(W.element("mult", L=1.0, n_slices=N, k1=0.5, k2=5.0,
                                                   split_order=order), gg)
            _, Sg, lg = st.track(ring, z0.reshape(6, 1), S0.reshape(3, 1), 1, 1)
            assert not lg.any()
            e.append(np.linalg.norm(Sg[:, 0] - Sref))
        assert all(lo < e[i] / e[i + 1] < hi for i in range(3)), (order, e)


def test_split_order_validation():
    with pytest.raises(st.SpinTrackError):
        st.Lattice(W.single_element_ring(W.element("sbend", L=1.0, n_slices=2, angle=0.1, split_order=4), 45.5))
    with pytest.raises(st.SpinTrackError):
        st.Lattice(W.single_element_ring(W.element("mult", L=1.0, n_slices=2, k1=0.1, split_order=3), 45.5))
    ring = W.with_split_order(W.with_spin_order(W.toy_ring(45.5), 2), 4)
    lat = st.Lattice(ring)
    st.Tracker(lat, 64, precision="mixed").close()
    st.Tracker(lat, 64).close()
    lat.close()


# ---- the mixed-precision tracker's fourth-order slices --------------------------

def spin_err(Sa, Sb):
    d = np.linalg.norm(Sa - Sb, axis=0)
    return float(d.mean()), float(d.max())


def mixed_vs_oracle(ring, z, S, turns, K):
    zm, Sm, lm = st.track(ring, z, S, turns, K, precision="mixed")
    zo, So, lo = oracle.track(ring, z, S, turns, K)
    assert np.array_equal(lm, lo)
    mean, mx = spin_err(Sm, So)
    assert mean < 1e-7 and mx < 1e-6, (mean, mx)
    assert np.abs(zm[:4] - zo[:4]).max() < 1e-8 and np.abs(zm[4] - zo[4]).max() < 1e-7


MIXED_ELEMENTS = ELEMENTS + [W.element("teapot", L=3.0, n_slices=8, angle=0.1, eta=0.98, fringe=1, split_order=4)]


@pytest.mark.parametrize("el", MIXED_ELEMENTS, ids=["dkd", "mk_f", "mk_d", "teapot"])
@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_mixed_single_fourth_order_element(el, K):
    """Fourth-order multipole, matrix-kick quadrupoles of both signs and a
    TEAPOT bend in the mixed-precision tracker, 10 passes against the oracle.
    These strong elements (k2 = 5 m^-3, 0.04 rad of spin rotation per pass in
    the quadrupole) are the mixed tracker's hardest single-element cases: its
    second-order slices already reach a mean Delta S of 1e-7 on them, so the
    fourth-order slices must stay within twice the second-order ones' error on
    the same element (or 1e-7), below 1e-6, with the orbit within 1e-8."""
    gg = 45.5
    z, S = W.gaussian_particles(257, gg, seed=190 + K)
    means = []
    for order in (4, 2):
        ring = W.single_element_ring(dict(el, split_order=order), gg)
        zm, Sm, lm = st.track(ring, z, S, 10, K, precision="mixed")
        zo, So, lo = oracle.track(ring, z, S, 10, K)
        assert np.array_equal(lm, lo)
        mean, mx = spin_err(Sm, So)
        assert mean < 1e-6 and mx < 1e-5, (order, mean, mx)
        assert np.abs(zm[:4] - zo[:4]).max() < 1e-8
        means.append(mean)
    assert means[0] <= max(2.0 * means[1], 1e-7), means


@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_mixed_rhic_like_rings_fourth_order(gg):
    ring = W.with_fringes(W.with_split_order(W.with_spin_order(W.rhic_like_ring(gg, n_cells=20), 2), 4))
    z, S = W.gaussian_particles(300, gg, seed=131)
    mixed_vs_oracle(ring, z, S, 10, 2)
    dk = W.with_split_order(W.with_spin_order(W.drift_kick_ring(W.rhic_like_ring(gg, n_cells=20)), 2), 4)
    mixed_vs_oracle(dk, z, S, 10, 2)


def test_mixed_fourth_order_1000_turns_within_1e_6():
    """1000 turns of the full RHIC-like ring with fourth-order quadrupole and
    sextupole slices at G gamma0 = 487: the mixed tracker against the FP64
    tracker, mean Delta S within 1e-6, orbit within 1e-6."""
    ring = W.with_split_order(W.with_spin_order(W.rhic_like_ring(487.0), 2), 4)
    z, S = W.gaussian_particles(1024, 487.0, seed=3453)
    zm, Sm, lm = st.track(ring, z, S, 1000, 2, precision="mixed")
    zf, Sf, lf = st.track(ring, z, S, 1000, 2)
    assert np.array_equal(lm, lf)
    mean, mx = spin_err(Sm, Sf)
    print(f"fourth-order ring at 487: mixed vs FP64 after 1000 turns: dS mean {mean:.3e} max {mx:.3e}")
    assert mean <= 1e-6, (mean, mx)
    assert np.abs(zm[:4] - zf[:4]).max() < 1e-6


def test_mixed_batched_jobs_fourth_order():
    rings = [W.with_split_order(W.with_spin_order(W.rhic_like_ring(gg, n_cells=c), 2), 4)
             for gg, c in ((45.5, 6), (300.0, 8))]
    rings.append(W.with_split_order(W.with_spin_order(W.drift_kick_ring(W.toy_ring(45.5)), 2), 4))
    rings.append(W.with_spin_order(W.toy_ring(45.5), 2))
    ns = [150, 97, 64, 33]
    b = st.Batch(rings, ns, "mixed")
    inputs = []
    for k, (ring, n) in enumerate(zip(rings, ns)):
        z, S = W.gaussian_particles(n, ring["Ggamma0"], seed=195 + k)
        b.upload(k, z, S)
        inputs.append((z, S))
    b.track(3, 2)
    for k, (ring, (z, S)) in enumerate(zip(rings, inputs)):
        zb, Sb, lb = b.download(k)
        zo, So, lo = oracle.track(ring, z, S, 3, 2)
        assert np.array_equal(lb, lo)
        mean, mx = spin_err(Sb, So)
        assert mean < 1e-7 and mx < 1e-6, (k, mean, mx)
        assert np.abs(zb[:4] - zo[:4]).max() < 1e-8
    b.close()
