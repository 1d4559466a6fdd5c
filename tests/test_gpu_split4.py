"""GPU parity of the fourth-order slice maps (Sec. 3.3: Yoshida's composition
of the symmetric drift-kick and matrix-kick maps of Eq. (27)): the CUDA FP64
tracker through the C ABI against the CPU oracle at 1e-11 for single
elements at every Romberg order, a RHIC-like ring with fourth-order maps and
fringe kicks, and the batched entry point; and the CUDA result's own rate of
convergence to the Thomas-BMT ODE through a strong multipole."""
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


def test_split_order_validation_and_mixed_rejection():
    with pytest.raises(st.SpinTrackError):
        st.Lattice(W.single_element_ring(W.element("sbend", L=1.0, n_slices=2, angle=0.1, split_order=4), 45.5))
    with pytest.raises(st.SpinTrackError):
        st.Lattice(W.single_element_ring(W.element("mult", L=1.0, n_slices=2, k1=0.1, split_order=3), 45.5))
    ring = W.with_split_order(W.with_spin_order(W.toy_ring(45.5), 2), 4)
    lat = st.Lattice(ring)
    with pytest.raises(st.SpinTrackError):
        st.Tracker(lat, 64, precision="mixed")
    st.Tracker(lat, 64).close()
    lat.close()
