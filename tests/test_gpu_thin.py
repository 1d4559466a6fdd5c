"""GPU parity of the thin lens (Sec. 3.5): the CUDA FP64 tracker through the C
ABI against the CPU oracle on the same seeded inputs, every coordinate and
spin component at 1e-11: single thin lenses at every Romberg order and both
midpoint schemes, the RHIC-like ring with thin sextupoles, batched jobs and
the allocation-free entry, lost particles, validation; and the mixed-precision
tracker on thin lenses within its error budget."""
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


def toy_with_thin_lenses(gg):
    """The toy ring with a thin sextupole-quadrupole lens in the middle of
    every drift after a quadrupole."""
    ring = W.toy_ring(gg)
    els = []
    for e in ring["elements"]:
        if e["type"] == "drift" and els and els[-1]["type"] == "mult":
            half = dict(e, L=0.5 * e["L"])
            sgn = 1.0 if els[-1]["k1"] > 0 else -1.0
            els += [half, W.element("thin_mult", n_slices=4, k1=0.002 * sgn, k2=0.3 * sgn), dict(half)]
        else:
            els.append(dict(e))
    return dict(ring, elements=els, name="toy_thin_lenses")


@pytest.mark.parametrize("gg", [45.5, 487.0])
@pytest.mark.parametrize("K", [0, 1, 2, 3, st.ST_SPIN_MID_HALF, st.ST_SPIN_MID_KICK])
def test_single_thin_lens(gg, K):
    el = W.element("thin_mult", n_slices=8, k1=0.05, k2=2.0)
    z, S = W.gaussian_particles(257, gg, seed=300 + K, sigmas=dict(x=3e-3, y=3e-3, px=3e-4, py=3e-4))
    zg, Sg, _ = compare(W.single_element_ring(el, gg), z, S, 10, K)
    assert np.array_equal(zg[[0, 2, 4, 5]], z[[0, 2, 4, 5]])        # positions, T, Pt untouched
    assert np.abs(Sg - S).max() > 1e-6


@pytest.mark.parametrize("K", [2, st.ST_SPIN_MID_KICK])
def test_toy_ring_with_thin_lenses(K):
    ring = toy_with_thin_lenses(45.5)
    z, S = W.gaussian_particles(500, 45.5, seed=41)
    compare(ring, z, S, 50, K)


def test_rhic_like_ring_with_thin_sextupoles():
    ring = W.with_spin_order(W.with_thin_sextupoles(W.rhic_like_ring(45.5)), 2)
    z, S = W.gaussian_particles(200, 45.5, seed=42)
    compare(ring, z, S, 3, 2)


def test_thin_lenses_in_batched_jobs_and_the_allocation_free_entry():
    import torch
    rings = [toy_with_thin_lenses(45.5), W.with_spin_order(W.with_thin_sextupoles(W.rhic_like_ring(300.0, n_cells=6)), 2)]
    ns = [200, 90]
    b = st.Batch(rings, ns, "fp64")
    inputs = []
    for k, (ring, n) in enumerate(zip(rings, ns)):
        z, S = W.gaussian_particles(n, ring["Ggamma0"], seed=90 + k)
        b.upload(k, z, S)
        inputs.append((z, S))
    b.track(4, 2)
    for k, (ring, (z, S)) in enumerate(zip(rings, inputs)):
        zb, Sb, lb = b.download(k)
        zo, So, lo = oracle.track(ring, z, S, 4, 2)
        assert np.array_equal(lb, lo)
        assert np.abs(zb - zo).max() < TOL and np.abs(Sb - So).max() < TOL
    b.close()
    ring = rings[0]
    z, S = inputs[0]
    n = z.shape[1]
    state = torch.from_numpy(st.pairs_from_soa(z, S)).to("cuda")
    lost = torch.zeros(n, dtype=torch.uint8, device="cuda")
    st.st_track_fp64_noalloc(ring["elements"], ring["G"], ring["Ggamma0"], state.data_ptr(), lost.data_ptr(), n, 5,
                             2, torch.cuda.current_stream().cuda_stream)
    za, Sa = st.soa_from_pairs(state.cpu().numpy(), n)
    zo, So, lo = oracle.track(ring, z, S, 5, 2)
    assert np.array_equal(lost.cpu().numpy(), lo)
    assert np.abs(za - zo).max() < TOL and np.abs(Sa - So).max() < TOL


def test_lost_in_a_thin_lens_keeps_entrance_state():
    gg = 45.5
    ring = toy_with_thin_lenses(gg)
    ring["elements"] = [e for e in ring["elements"] if e["type"] == "thin_mult"][:1] + ring["elements"]
    z, S = W.gaussian_particles(40, gg, seed=5)
    # at X = 2 m the lens kicks Px by about -0.6: from -0.9 past -1, so Ps
    # turns imaginary inside the first thin lens
    z[0, 11], z[1, 11], z[5, 11] = 2.0, -0.9, 0.0
    zg, Sg, lg = compare(ring, z, S, 2, 2)
    assert lg[11] == 1 and lg.sum() == 1
    assert np.array_equal(zg[:, 11], z[:, 11]) and np.array_equal(Sg[:, 11], S[:, 11])


def spin_err(Sa, Sb):
    d = np.linalg.norm(Sa - Sb, axis=0)
    return float(d.mean()), float(d.max())


def test_mixed_tracker_with_thin_lenses_against_the_oracle():
    """The mixed-precision tracker runs thin lenses as drift-less multipoles:
    on the toy ring with thin lenses after 100 turns its spins stay within
    1e-7 (mean) and 1e-6 (max) of the oracle, its transverse orbit within
    1e-7, as on the toy ring without them."""
    ring = toy_with_thin_lenses(45.5)
    z, S = W.gaussian_particles(512, 45.5, seed=7)
    zm, Sm, lm = st.track(ring, z, S, 100, 2, precision="mixed")
    zo, So, lo = oracle.track(ring, z, S, 100, 2)
    assert np.array_equal(lm, lo)
    mean, mx = spin_err(Sm, So)
    assert mean < 1e-7 and mx < 1e-6, (mean, mx)
    assert np.abs(zm[:4] - zo[:4]).max() < 1e-7


@pytest.mark.parametrize("gg", [487.0])   # the larger spin rotation per turn
def test_mixed_tracker_thin_sextupole_ring_1000_turns(gg):
    """The mixed tracker's error bound on the RHIC-like ring with thin
    sextupoles: after 1000 turns the mean spin error over 1024 particles
    against the FP64 tracker stays within 1e-6."""
    ring = W.with_spin_order(W.with_thin_sextupoles(W.rhic_like_ring(gg)), 2)
    z, S = W.gaussian_particles(1024, gg, seed=3451)
    zm, Sm, lm = st.track(ring, z, S, 1000, 2, precision="mixed")
    zf, Sf, lf = st.track(ring, z, S, 1000, 2, precision="fp64")
    assert np.array_equal(lm, lf)
    mean, mx = spin_err(Sm, Sf)
    assert mean <= 1e-6, (mean, mx)
    assert np.abs(zm[:4] - zf[:4]).max() < 1e-6


def test_thin_lens_validation():
    ring = toy_with_thin_lenses(45.5)
    lat = st.Lattice(ring)
    st.Tracker(lat, 64, precision="mixed").close()
    st.Tracker(lat, 64).close()
    lat.close()
    for bad in (dict(L=0.1), dict(fringe=1), dict(split_order=4)):
        el = dict(W.element("thin_mult", n_slices=4, k2=1.0), **bad)
        with pytest.raises(st.SpinTrackError):
            st.Lattice(W.single_element_ring(el, 45.5))


@pytest.mark.parametrize("K", [0, 4, st.ST_SPIN_MID_KICK])
def test_extreme_slice_counts(K):
    """One slice everywhere (midpoint and trapezoid) and the largest slice
    count of the boundary (4096) on a thin lens, a TEAPOT bend and a
    multipole.  The oracle's TEAPOT bend rounds X to about an ulp of 1/h in
    each of its 8192 printed-form curved drifts (1.4e-11 from its long-double
    build here), so that element is held to the long-double oracle as closely
    as the FP64 oracle is."""
    gg = 45.5
    z, S = W.gaussian_particles(64, gg, seed=12)
    if K in (0, st.ST_SPIN_MID_KICK):
        ring = W.with_slices(toy_with_thin_lenses(gg), 1)
        compare(ring, z, S, 5, K)
        compare(W.with_slices(W.drift_kick_ring(W.toy_ring(gg)), 1), z, S, 3, K)
    for el in (W.element("thin_mult", n_slices=4096, k1=0.02, k2=1.0),
               W.element("mult", L=0.5, n_slices=4096, k1=0.1, k2=2.0)):
        compare(W.single_element_ring(el, gg), z, S, 1, K)
    ring = W.single_element_ring(W.element("teapot", L=3.0, n_slices=4096, angle=0.2), gg)
    zg, Sg, lg = st.track(ring, z, S, 1, K)
    zo, So, lo = oracle.track(ring, z, S, 1, K)
    zx, Sx, lx = oracle.track(ring, z, S, 1, K, variant="f80")
    zx, Sx = zx.astype(np.float64), Sx.astype(np.float64)
    assert np.array_equal(lg, lx) and np.array_equal(lo, lx)
    assert np.abs(zg - zx).max() < 2.0 * np.abs(zo - zx).max() + 1e-14
    assert np.abs(Sg - Sx).max() < 2.0 * np.abs(So - Sx).max() + 1e-13


def test_mixed_batch_with_thin_lenses():
    """Thin-lens rings in one mixed-precision batch: each job within the
    mixed tracker's budget of the oracle after 20 turns."""
    rings = [toy_with_thin_lenses(45.5), W.with_spin_order(W.with_thin_sextupoles(W.rhic_like_ring(120.0, n_cells=6)), 2)]
    ns = [256, 100]
    b = st.Batch(rings, ns, "mixed")
    inputs = []
    for k, (ring, n) in enumerate(zip(rings, ns)):
        z, S = W.gaussian_particles(n, ring["Ggamma0"], seed=95 + k)
        b.upload(k, z, S)
        inputs.append((z, S))
    b.track(20, 2)
    for k, (ring, (z, S)) in enumerate(zip(rings, inputs)):
        zb, Sb, lb = b.download(k)
        zo, So, lo = oracle.track(ring, z, S, 20, 2)
        assert np.array_equal(lb, lo)
        mean, mx = spin_err(Sb, So)
        assert mean < 1e-7 and mx < 1e-6, (k, mean, mx)
        assert np.abs(zb[:4] - zo[:4]).max() < 1e-7
    b.close()
