"""GPU parity of the thin dipole and multipole fringe spin kicks (Sec. 4.5,
Eq. (skfringe)): the CUDA FP64 tracker through the C ABI against the CPU
oracle on the same seeded inputs, every coordinate and spin component at
1e-11, for single elements with fringes at every Romberg order, RHIC-like
rings with fringe kicks on every magnet, lost particles, the batched entry
point and the flag's validation; and the mixed-precision tracker's kicks
within its error budget."""
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


ELEMENTS = [
    W.element("quad_mk", L=1.0, n_slices=8, k1=0.3, fringe=1),
    W.element("mult", L=1.0, n_slices=8, k1=-0.2, k2=5.0, fringe=1),
    W.element("sbend", L=3.0, n_slices=8, angle=0.05, fringe=1),
]


@pytest.mark.parametrize("el", ELEMENTS, ids=lambda e: e["type"])
@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_single_element_with_fringes_every_order(el, K):
    gg = 45.5
    ring = W.single_element_ring(el, gg)
    z, S = W.gaussian_particles(257, gg, seed=70 + K, sigmas=dict(x=3e-3, y=3e-3))
    zg, Sg, lg = compare(ring, z, S, 10, K)
    # the kicks change the result
    _, Sn, _ = st.track(W.with_fringes(ring, 0), z, S, 10, K)
    assert np.abs(Sg - Sn).max() > 1e-9


@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_rhic_like_ring_with_fringes(gg):
    ring = W.with_fringes(W.with_spin_order(W.rhic_like_ring(gg, n_cells=20), 2))
    z, S = W.gaussian_particles(300, gg, seed=8)
    compare(ring, z, S, 10, 2)


def test_toy_ring_with_fringes_100_turns():
    ring = W.with_fringes(W.with_spin_order(W.toy_ring(45.5), 2))
    z, S = W.gaussian_particles(500, 45.5, seed=12)
    compare(ring, z, S, 100, 2)


def test_lost_in_an_element_with_fringes_keeps_entrance_state():
    ring = W.with_fringes(W.with_spin_order(W.toy_ring(45.5), 2))
    z, S = W.gaussian_particles(64, 45.5, seed=9)
    z[1, 5] = 1.5          # lost in the first slice of the first quadrupole
    z[3, 40] = -1.2
    zg, Sg, lg = compare(ring, z, S, 2, 2)
    assert lg[5] == 1 and lg[40] == 1 and lg.sum() == 2
    assert np.array_equal(zg[:, 5], z[:, 5]) and np.array_equal(Sg[:, 40], S[:, 40])


def test_batched_jobs_with_fringes():
    rings = [W.with_fringes(W.with_spin_order(W.rhic_like_ring(gg, n_cells=c), 2)) for gg, c in ((45.5, 6), (200.0, 10))]
    rings.append(W.with_spin_order(W.toy_ring(45.5), 2))
    ns = [200, 333, 64]
    b = st.Batch(rings, ns, "fp64")
    inputs = []
    for k, (ring, n) in enumerate(zip(rings, ns)):
        z, S = W.gaussian_particles(n, ring["Ggamma0"], seed=80 + k)
        b.upload(k, z, S)
        inputs.append((z, S))
    b.track(3, 2)
    for k, (ring, (z, S)) in enumerate(zip(rings, inputs)):
        zb, Sb, lb = b.download(k)
        zo, So, lo = oracle.track(ring, z, S, 3, 2)
        assert np.array_equal(lb, lo)
        assert np.abs(zb - zo).max() < TOL and np.abs(Sb - So).max() < TOL
    b.close()


def test_fringe_flag_validation():
    with pytest.raises(st.SpinTrackError):
        st.Lattice(W.single_element_ring(W.element("drift", L=1.0, fringe=1), 45.5))
    with pytest.raises(st.SpinTrackError):
        st.Lattice(W.single_element_ring(W.element("snake", snake_mu=np.pi, fringe=1), 45.5))
    with pytest.raises(st.SpinTrackError):
        st.Lattice(W.single_element_ring(W.element("mult", L=1.0, n_slices=4, k1=0.1, fringe=2), 45.5))


def spin_err(Sa, Sb):
    d = np.linalg.norm(Sa - Sb, axis=0)
    return float(d.mean()), float(d.max())


def test_mixed_tracker_with_fringe_kicks_against_the_oracle():
    """The mixed-precision tracker applies the fringe kicks as near-identity
    rotations about s around its element rotations: on the toy ring with
    fringe kicks on every magnet after 100 turns its spins stay within 1e-7
    (mean) and 1e-6 (max) of the oracle, as without kicks."""
    ring = W.with_fringes(W.with_spin_order(W.toy_ring(45.5), 2))
    z, S = W.gaussian_particles(512, 45.5, seed=17)
    zm, Sm, lm = st.track(ring, z, S, 100, 2, precision="mixed")
    zo, So, lo = oracle.track(ring, z, S, 100, 2)
    assert np.array_equal(lm, lo)
    mean, mx = spin_err(Sm, So)
    assert mean < 1e-7 and mx < 1e-6, (mean, mx)
    assert np.abs(zm[:4] - zo[:4]).max() < 1e-7
    # the kicks matter at this level: without them the oracle differs by more
    _, Sp, _ = oracle.track(W.with_fringes(ring, 0), z, S, 100, 2)
    assert spin_err(Sp, So)[0] > 100 * mean


@pytest.mark.parametrize("gg", [487.0])   # the larger spin rotation per turn
def test_mixed_tracker_with_fringe_kicks_1000_turns(gg):
    """The mixed tracker's error bound on the RHIC-like ring with fringe kicks
    on every magnet: after 1000 turns the mean spin error over 1024
    particles against the FP64 tracker stays within 1e-6."""
    ring = W.with_fringes(W.with_spin_order(W.rhic_like_ring(gg), 2))
    z, S = W.gaussian_particles(1024, gg, seed=3451)
    zm, Sm, lm = st.track(ring, z, S, 1000, 2, precision="mixed")
    zf, Sf, lf = st.track(ring, z, S, 1000, 2, precision="fp64")
    assert np.array_equal(lm, lf)
    mean, mx = spin_err(Sm, Sf)
    assert mean <= 1e-6, (mean, mx)
    assert np.abs(zm[:4] - zf[:4]).max() < 1e-6


def test_mixed_batch_and_orbit_only_with_fringe_kicks():
    """A mixed batch of a ring with fringe kicks and one without (the fringe
    instantiation decodes both), and orbit-only mixed tracking of the kicked
    ring (the kicks leave the orbit alone)."""
    rings = [W.with_fringes(W.with_spin_order(W.toy_ring(45.5), 2)), W.with_spin_order(W.toy_ring(120.0), 2)]
    ns = [200, 90]
    b = st.Batch(rings, ns, "mixed")
    inputs = []
    for k, (ring, n) in enumerate(zip(rings, ns)):
        z, S = W.gaussian_particles(n, ring["Ggamma0"], seed=60 + k)
        b.upload(k, z, S)
        inputs.append((z, S))
    b.track(20, 2)
    for k, (ring, (z, S)) in enumerate(zip(rings, inputs)):
        zb, Sb, lb = b.download(k)
        zo, So, lo = oracle.track(ring, z, S, 20, 2)
        assert np.array_equal(lb, lo)
        mean, mx = spin_err(Sb, So)
        assert mean < 1e-7 and mx < 1e-6, (k, mean, mx)
    b.close()
    ring = rings[0]
    z, S = inputs[0]
    lat = st.Lattice(ring)
    t = st.Tracker(lat, z.shape[1], precision="mixed")
    t.upload(z, S)
    t.track_orbit(20)
    zm, Sm, _ = t.download()
    t.close()
    lat.close()
    zp, _, _ = st.track(W.with_fringes(ring, 0), z, S, 20, 2, precision="mixed")
    assert np.array_equal(Sm, S)
    assert np.abs(zm[:4] - zp[:4]).max() < 1e-9      # the same maps, compiled apart (mixed arithmetic)
