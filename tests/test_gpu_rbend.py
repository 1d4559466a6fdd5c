"""GPU parity of the rectangular bend (Sec. 3.2: dynamic rotations, thin-fringe
orbit maps, exact body map, offsets; Sec. 4.5: fringe spin kicks of Eq.
(skfringeRB)): the CUDA FP64 tracker through the C ABI against the CPU oracle
on the same seeded inputs, every coordinate and spin component at 1e-11, for
single magnets at every Romberg order (symmetric and asymmetric faces, field
errors, with and without fringe kicks), a ring of rectangular bends, the
reference particle's closed form, lost particles, batched jobs, validation and
the mixed tracker's refusal."""
import math

import numpy as np
import pytest

import oracle
import paper_1501_03450_b300 as st
import workloads as W

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


MAGNETS = [
    dict(e1=0.0, eta=1.0, fringe=0),
    dict(e1=0.012, eta=1.0, fringe=1),
    dict(e1=-0.007, eta=1.003, fringe=1),
]


@pytest.mark.parametrize("kw", MAGNETS, ids=["symmetric", "asymmetric_kicks", "field_error"])
@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_single_rectangular_bend_every_order(kw, K):
    gg = 45.5
    el = W.element("rbend", L=3.0, n_slices=8, angle=0.06, **kw)
    ring = W.single_element_ring(el, gg)
    z, S = W.gaussian_particles(257, gg, seed=120 + K, sigmas=dict(x=3e-3, y=3e-3, px=3e-4, py=3e-4))
    compare(ring, z, S, 10, K)


def test_reference_particle_closed_form():
    """On-axis particle: back on the axis with T = 0, spin turned by
    -G gamma0 * angle about y."""
    gg, ang = 487.0, 0.05
    ring = W.single_element_ring(W.element("rbend", L=3.0, n_slices=8, angle=ang, e1=0.01), gg)
    z = np.zeros((6, 1))
    S = np.array([[0.0], [0.0], [1.0]])
    zg, Sg, lg = st.track(ring, z, S, 1, 2)
    assert np.abs(zg).max() < 5e-15
    th = -gg * ang
    np.testing.assert_allclose(Sg[:, 0], [math.sin(th), 0.0, math.cos(th)], rtol=0, atol=1e-12)


@pytest.mark.parametrize("fringe", [0, 1])
def test_ring_of_rectangular_bends_100_turns(fringe):
    ring = W.with_spin_order(W.rbend_ring(45.5, fringe=fringe), 2)
    z, S = W.gaussian_particles(400, 45.5, seed=33)
    compare(ring, z, S, 100, 2)


def test_ring_of_rectangular_bends_high_energy():
    ring = W.with_spin_order(W.rbend_ring(487.0, e1=0.005, fringe=1), 2)
    z, S = W.gaussian_particles(200, 487.0, seed=34)
    compare(ring, z, S, 4, 2)


def test_lost_in_a_rectangular_bend_keeps_entrance_state():
    ring = W.with_spin_order(W.rbend_ring(45.5), 2)
    ring["elements"] = ring["elements"][2:] + ring["elements"][:2]     # a bend first
    assert ring["elements"][0]["type"] == "rbend"
    z, S = W.gaussian_particles(40, 45.5, seed=35)
    z[1, 7] = 1.2          # no real longitudinal momentum
    z[1, 20] = 0.985       # moving nearly parallel to the entrance face: never reaches it
    zg, Sg, lg = compare(ring, z, S, 2, 2)
    assert lg[7] == 1 and lg[20] == 1 and lg.sum() == 2
    assert np.array_equal(zg[:, 7], z[:, 7]) and np.array_equal(Sg[:, 20], S[:, 20])


def test_batched_jobs_with_rectangular_bends():
    rings = [W.with_spin_order(W.rbend_ring(gg, fringe=f), 2) for gg, f in ((45.5, 1), (150.0, 0))]
    rings.append(W.with_spin_order(W.toy_ring(45.5), 2))
    ns = [200, 90, 64]
    b = st.Batch(rings, ns, "fp64")
    inputs = []
    for k, (ring, n) in enumerate(zip(rings, ns)):
        z, S = W.gaussian_particles(n, ring["Ggamma0"], seed=130 + k)
        b.upload(k, z, S)
        inputs.append((z, S))
    b.track(3, 2)
    for k, (ring, (z, S)) in enumerate(zip(rings, inputs)):
        zb, Sb, lb = b.download(k)
        zo, So, lo = oracle.track(ring, z, S, 3, 2)
        assert np.array_equal(lb, lo)
        assert np.abs(zb - zo).max() < TOL and np.abs(Sb - So).max() < TOL
    b.close()


def test_rbend_validation_and_mixed_rejection():
    for el in (W.element("rbend", L=2.0, n_slices=4, angle=0.0),
               W.element("rbend", L=2.0, n_slices=4, angle=0.1, eta=0.0),
               W.element("rbend", L=2.0, n_slices=4, angle=0.1, e1=1.6)):
        with pytest.raises(st.SpinTrackError):
            st.Lattice(W.single_element_ring(el, 45.5))
    ring = W.with_spin_order(W.rbend_ring(45.5), 2)
    lat = st.Lattice(ring)
    with pytest.raises(st.SpinTrackError):
        st.Tracker(lat, 64, precision="mixed")
    st.Tracker(lat, 64).close()
    lat.close()
