"""Mixed-precision tracker (FP32 slices with compensated coordinates, FP64
per-turn spin composition) through the C ABI, against the CPU oracle and
against the FP64 GPU tracker (itself pinned to the oracle at 1e-11).

The mixed tracker computes the same discretisation as the FP64 one in a
different arithmetic, so the comparison is an error budget, not bit parity.
Metric: Delta S = mean_j |S_j - S_j(ref)| (Sec. 5.2.2), with the maximum also
bounded, and the max absolute orbit error."""
import numpy as np
import pytest

import oracle
import paper_1501_03450_b300 as st
import workloads as W

pytestmark = pytest.mark.gpu


# measured at G gamma0 = 487 (1024 particles, 1000 turns): p50 4.8e-8, p90 6.0e-7,
# p99 2.5e-6, max 7.4e-6
TAIL_P99_487 = 8e-6
TAIL_MAX_487 = 2.5e-5


def spin_err(Sa, Sb):
    d = np.linalg.norm(Sa - Sb, axis=0)
    return float(d.mean()), float(d.max())


def test_toy_ring_mixed_vs_oracle_100_turns():
    w = W.workload("toy_ring_1024")
    z, S = W.gaussian_particles(1024, 45.5, seed=w["seed"])
    zm, Sm, lm = st.track(w["ring"], z, S, 100, 2, precision="mixed")
    zo, So, lo = oracle.track(w["ring"], z, S, 100, 2)
    assert np.array_equal(lm, lo)
    mean, mx = spin_err(Sm, So)
    assert mean < 1e-7 and mx < 1e-6, (mean, mx)
    assert np.abs(zm[:4] - zo[:4]).max() < 1e-7
    assert np.abs(zm[4] - zo[4]).max() < 1e-5          # T is passive; FP32 path-length terms


@pytest.mark.parametrize("gg,mean_tol,max_tol", [(45.5, 1e-8, 1e-7), (487.0, 3e-7, 1e-5)])
def test_rhic_like_ring_mixed_100_turns(gg, mean_tol, max_tol):
    ring = W.with_spin_order(W.rhic_like_ring(gg), 2)
    z, S = W.gaussian_particles(512, gg, seed=3451)
    zm, Sm, _ = st.track(ring, z, S, 100, 2, precision="mixed")
    zf, Sf, _ = st.track(ring, z, S, 100, 2, precision="fp64")
    mean, mx = spin_err(Sm, Sf)
    assert mean < mean_tol and mx < max_tol, (mean, mx)
    assert np.abs(zm[:4] - zf[:4]).max() < 3e-7


def test_rhic_like_ring_mixed_vs_oracle_direct():
    ring = W.with_spin_order(W.rhic_like_ring(45.5), 2)
    z, S = W.gaussian_particles(64, 45.5, seed=77)
    zm, Sm, _ = st.track(ring, z, S, 5, 2, precision="mixed")
    zo, So, _ = oracle.track(ring, z, S, 5, 2)
    mean, mx = spin_err(Sm, So)
    assert mean < 1e-7 and mx < 1e-6
    assert np.abs(zm[:4] - zo[:4]).max() < 1e-9


@pytest.mark.parametrize("K", [0, 1, 2, 3, 4])
def test_mixed_every_romberg_order(K):
    ring = W.with_spin_order(W.toy_ring(45.5), K)
    z, S = W.gaussian_particles(200, 45.5, seed=30 + K)
    zm, Sm, _ = st.track(ring, z, S, 10, K, precision="mixed")
    zo, So, _ = oracle.track(ring, z, S, 10, K)
    mean, mx = spin_err(Sm, So)
    assert mean < 1e-7 and mx < 1e-6, (K, mean, mx)
    assert np.abs(zm[:4] - zo[:4]).max() < 1e-8


def test_mixed_full_size_sampled():
    """10^6 particles (the mixed-precision workload's size) for 2 turns;
    256 particles sampled across the ensemble against the oracle."""
    ring = W.with_spin_order(W.rhic_like_ring(45.5), 2)
    n = 1_000_000
    z, S = W.gaussian_particles(n, 45.5, seed=3451)
    zm, Sm, lm = st.track(ring, z, S, 2, 2, precision="mixed")
    idx = np.linspace(0, n - 1, 256).astype(int)
    zo, So, lo = oracle.track(ring, z[:, idx], S[:, idx], 2, 2)
    assert np.array_equal(lm[idx], lo)
    mean, mx = spin_err(Sm[:, idx], So)
    assert mean < 1e-7 and mx < 1e-6
    assert np.abs(zm[:4, idx] - zo[:4]).max() < 1e-9


def test_mixed_lost_particle_and_edge_cases():
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    z, S = W.gaussian_particles(33, 45.5, seed=3)
    z[1, 5] = 1.5                       # lost in the first element
    z[:, 0] = 0.0                       # on axis: zero-angle edge rotations
    zm, Sm, lm = st.track(ring, z, S, 3, 2, precision="mixed")
    zo, So, lo = oracle.track(ring, z, S, 3, 2)
    assert np.array_equal(lm, lo) and lm[5] == 1
    assert np.abs(zm - zo).max() < 1e-6
    assert spin_err(Sm, So)[1] < 1e-6


@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_mixed_spin_error_1000_turns_within_1e_6(gg):
    """The stated bound: after 1000 turns on the RHIC-like ring, the mean spin
    error of the mixed tracker over 1024 particles against the FP64 tracker
    (which matches the oracle to 1e-11) stays within 1e-6."""
    ring = W.with_spin_order(W.rhic_like_ring(gg), 2)
    z, S = W.gaussian_particles(1024, gg, seed=3451)
    zm, Sm, lm = st.track(ring, z, S, 1000, 2, precision="mixed")
    zf, Sf, lf = st.track(ring, z, S, 1000, 2, precision="fp64")
    assert np.array_equal(lm, lf)
    mean, mx = spin_err(Sm, Sf)
    d = np.linalg.norm(Sm - Sf, axis=0)
    p50, p90, p99 = np.percentile(d, [50, 90, 99])
    print(f"mixed vs FP64 after 1000 turns at {gg}: dS mean {mean:.3e} p50 {p50:.3e} p90 {p90:.3e} "
          f"p99 {p99:.3e} max {mx:.3e}")
    assert mean <= 1e-6, (mean, mx)
    assert np.abs(zm[:4] - zf[:4]).max() < 1e-6
    # the tail: every particle within 1e-6 at 45.5; at 487, where a 1e-12 change
    # of Pt moves the FP64 tracker's own spins by 5e-7 on average, bounds with
    # a margin of about 3 over the measured p99 and max
    if gg < 100.0:
        assert mx <= 1e-6, mx
    else:
        assert p99 <= TAIL_P99_487 and mx <= TAIL_MAX_487, (p99, mx)


def test_mixed_orbit_only_tracks_the_mixed_orbit():
    """st_track_orbit on a mixed context: the mixed tracker's compensated orbit
    maps without the spin step (spins untouched), agreeing with the full mixed
    tracker's orbit and with the FP64 orbit."""
    ring = W.with_spin_order(W.rhic_like_ring(487.0, n_cells=20), 2)
    z, S = W.gaussian_particles(700, 487.0, seed=41)
    lat = st.Lattice(ring)
    tr = st.Tracker(lat, z.shape[1], "mixed")
    tr.upload(z, S)
    tr.track_orbit(10)
    zo, So, lo = tr.download()
    tr.close()
    lat.close()
    np.testing.assert_array_equal(So, S)
    zm, _, lm = st.track(ring, z, S, 10, 2, precision="mixed")
    zf, _, lf = st.track(ring, z, S, 10, 2, precision="fp64")
    assert np.array_equal(lo, lm) and np.array_equal(lo, lf)
    # the two kernels inline the same maps but may contract FP32 operations
    # differently: agreement to the mixed orbit's own accuracy
    assert np.abs(zo[:4] - zm[:4]).max() < 1e-9
    assert np.abs(zo[:4] - zf[:4]).max() < 1e-9


def test_mixed_stroboscopic_average_is_the_sum_of_the_turn_spins():
    """st_track_average on a mixed-precision context: the accumulated spin is
    the sum of the spins after each turn, bit for bit against tracking turn
    by turn in the same launch shape, and close to the FP64 tracker's average."""
    torch = pytest.importorskip("torch")
    ring = W.with_spin_order(W.rhic_like_ring(487.0, n_cells=12), 2)
    n, T = 333, 12
    z, S = W.gaussian_particles(n, 487.0, seed=77)
    lat = st.Lattice(ring)
    acc = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()                 # the tracker runs on its own stream
    tr = st.Tracker(lat, n, "mixed")
    tr.set_launch(block_threads=128, turns_per_launch=1)
    tr.upload(z, S)
    st.st_track_average(tr.handle, T, 2, acc.data_ptr())
    zA, SA, _ = tr.download()
    tr.upload(z, S)
    manual = np.zeros((3, n))
    for _ in range(T):
        tr.track(1, 2)
        _, Si, _ = tr.download()
        manual += Si
    zB, SB, _ = tr.download()
    tr.close()
    torch.cuda.synchronize()
    assert np.array_equal(zA, zB) and np.array_equal(SA, SB)
    assert np.array_equal(acc.cpu().numpy(), manual)
    acc64 = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    tr = st.Tracker(lat, n, "fp64")
    tr.upload(z, S)
    st.st_track_average(tr.handle, T, 2, acc64.data_ptr())
    tr.download()                            # synchronises the tracker's stream
    tr.close()
    lat.close()
    assert np.abs(acc.cpu().numpy() - acc64.cpu().numpy()).max() / T < 1e-6


@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_mixed_against_the_oracle_on_the_configured_subset(gg):
    """The mixed-precision configuration's error statement taken literally:
    1024 particles of the 10^6-particle ensemble (the first 1024, as the
    bench's subset), 1000 turns of the RHIC-like ring, the mixed tracker
    against the FP64 CPU oracle itself.  The oracle's own rounding noise after
    1000 turns (about 2e-8 in the spin at G*gamma0 = 487, against its
    long-double build) is far below the bound, so the comparison measures the
    mixed arithmetic: mean Delta S <= 1e-6, max below 1e-4, orbit below 1e-6 m."""
    ring = W.with_spin_order(W.rhic_like_ring(gg), 2)
    z, S = W.gaussian_particles(1024, gg, seed=3451)
    zm, Sm, lm = st.track(ring, z, S, 1000, 2, precision="mixed")
    zo, So, lo = oracle.track(ring, z, S, 1000, 2)
    assert np.array_equal(lm, lo) and lm.sum() == 0
    mean, mx = spin_err(Sm, So)
    print(f"G*gamma0={gg}: mixed vs oracle after 1000 turns: dS mean {mean:.3e} max {mx:.3e}, "
          f"orbit max {np.abs(zm[:5] - zo[:5]).max(axis=1)}")
    assert mean <= 1e-6 and mx < 1e-4, (mean, mx)
    assert np.abs(zm[:4] - zo[:4]).max() < 1e-6


MID = [st.ST_SPIN_MID_HALF, st.ST_SPIN_MID_KICK]


@pytest.mark.parametrize("K", MID)
@pytest.mark.parametrize("case", ["toy", "rhic_like_487", "thin_sextupoles", "fringes", "odd_slices"])
def test_mixed_midpoint_schemes_against_the_oracle(case, K):
    """The midpoint spin schemes (Sec. 4.1, Eq. (37)) in the mixed-precision
    tracker against the oracle's, on rings of every element kind the mixed
    tracker runs: the toy ring (drift-kick-drift quadrupoles, sector bends),
    the RHIC-like ring at G*gamma0 = 487 (matrix-kick quadrupoles,
    sextupoles, snakes), thin sextupoles, fringe spin kicks on every magnet,
    and three slices per element (the midpoint schemes take any n_slices).
    The same error budget as the mixed tracker's Romberg orders."""
    if case == "toy":
        ring, gg, turns = W.toy_ring(45.5), 45.5, 20
    elif case == "rhic_like_487":
        ring, gg, turns = W.with_spin_order(W.rhic_like_ring(487.0, n_cells=20), 2), 487.0, 10
    elif case == "thin_sextupoles":
        ring, gg, turns = W.with_thin_sextupoles(W.with_spin_order(W.rhic_like_ring(45.5, n_cells=12), 2)), 45.5, 10
    elif case == "fringes":
        ring, gg, turns = W.with_fringes(W.with_spin_order(W.rhic_like_ring(487.0, n_cells=12), 2)), 487.0, 10
    else:
        ring, gg, turns = W.with_slices(W.rhic_like_ring(45.5, n_cells=12), 3), 45.5, 10
    z, S = W.gaussian_particles(200, gg, seed=61)
    zm, Sm, lm = st.track(ring, z, S, turns, K, precision="mixed")
    zo, So, lo = oracle.track(ring, z, S, turns, K)
    assert np.array_equal(lm, lo)
    mean, mx = spin_err(Sm, So)
    assert mean < 1e-7 and mx < 1e-6, (case, K, mean, mx)
    assert np.abs(zm[:4] - zo[:4]).max() < 1e-8


@pytest.mark.parametrize("K", MID)
def test_mixed_midpoint_1000_turns_within_1e_6(K):
    """1000 turns of the RHIC-like ring at G*gamma0 = 487 with a midpoint
    scheme: the mixed tracker against the FP64 tracker with the same scheme
    (itself at parity with the oracle), mean Delta S within 1e-6."""
    ring = W.with_spin_order(W.rhic_like_ring(487.0), 2)
    z, S = W.gaussian_particles(1024, 487.0, seed=3451)
    zm, Sm, lm = st.track(ring, z, S, 1000, K, precision="mixed")
    zf, Sf, lf = st.track(ring, z, S, 1000, K)
    assert np.array_equal(lm, lf)
    mean, mx = spin_err(Sm, Sf)
    print(f"midpoint scheme {K}: mixed vs FP64 after 1000 turns at 487: dS mean {mean:.3e} max {mx:.3e}")
    assert mean <= 1e-6, (mean, mx)
    assert np.abs(zm[:4] - zf[:4]).max() < 1e-6


def test_mixed_midpoint_lost_particles_and_average():
    """A particle lost in the first element is flagged as by the oracle; the
    stroboscopic sum with a midpoint scheme is the sum of the turn spins (a
    lost particle adds its spin of the turn that lost it, and nothing after)."""
    torch = pytest.importorskip("torch")
    ring = W.toy_ring(45.5)
    z, S = W.gaussian_particles(40, 45.5, seed=62)
    z[1, 9] = 1.5
    zm, Sm, lm = st.track(ring, z, S, 3, st.ST_SPIN_MID_HALF, precision="mixed")
    zo, So, lo = oracle.track(ring, z, S, 3, st.ST_SPIN_MID_HALF)
    assert np.array_equal(lm, lo) and lm[9] == 1
    assert spin_err(Sm, So)[1] < 1e-6
    lat = st.Lattice(ring)
    acc = torch.zeros((3, 40), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    tr = st.Tracker(lat, 40, "mixed")
    tr.set_launch(block_threads=128, turns_per_launch=1)
    tr.upload(z, S)
    st.st_track_average(tr.handle, 5, st.ST_SPIN_MID_KICK, acc.data_ptr())
    _, SA, _ = tr.download()
    tr.upload(z, S)
    manual = np.zeros((3, 40))
    for turn in range(5):
        tr.track(1, st.ST_SPIN_MID_KICK)
        _, Si, li = tr.download()
        manual += Si
        if turn == 0:
            S_first = Si.copy()
    tr.close()
    lat.close()
    torch.cuda.synchronize()
    got = acc.cpu().numpy()
    alive = li == 0
    assert li[9] == 1 and alive.sum() == 39
    assert np.array_equal(got[:, alive], manual[:, alive])
    assert np.array_equal(got[:, 9], S_first[:, 9])


# ---- TEAPOT bends (Sec. 3.6) in the mixed-precision tracker -------------------

def mixed_vs_oracle(ring, z, S, turns, K, mean_tol=1e-7, max_tol=1e-6, orbit_tol=1e-8):
    zm, Sm, lm = st.track(ring, z, S, turns, K, precision="mixed")
    zo, So, lo = oracle.track(ring, z, S, turns, K)
    assert np.array_equal(lm, lo)
    alive = lo == 0
    mean, mx = spin_err(Sm[:, alive], So[:, alive])
    dz = np.abs(zm[:, alive] - zo[:, alive]).max(axis=1)
    assert mean < mean_tol and mx < max_tol, (mean, mx)
    assert dz[:4].max() < orbit_tol and dz[4] < 10 * orbit_tol, dz
    return zm, Sm, lm


TEAPOTS = [
    dict(eta=1.0, fringe=0),
    dict(eta=0.98, fringe=1),
    dict(eta=0.0, fringe=0),
]


@pytest.mark.parametrize("kw", TEAPOTS, ids=["design", "field_error_kicks", "field_free"])
@pytest.mark.parametrize("K", [0, 1, 2, 3, st.ST_SPIN_MID_HALF, st.ST_SPIN_MID_KICK])
def test_mixed_single_teapot_bend(kw, K):
    """One TEAPOT bend (design field, field error with fringe kicks, field-free
    curved frame) with every Romberg order and both midpoint schemes, 10
    turns, against the oracle.  In the field-free frame the particles leave
    the axis (a straight line in a frame that turns 0.1 rad per pass: X of
    order 0.1 m after one pass), outside the paraxial regime the mixed
    tracker is built for, so that case runs one pass with an orbit bound of
    1e-7 m."""
    gg = 45.5
    el = W.element("teapot", L=3.0, n_slices=8, angle=0.1, **kw)
    ring = W.single_element_ring(el, gg)
    z, S = W.gaussian_particles(257, gg, seed=300 + K, sigmas=dict(x=3e-3, y=3e-3, px=3e-4, py=3e-4))
    if kw["eta"] == 0.0:
        mixed_vs_oracle(ring, z, S, 1, K, orbit_tol=1e-7)
    else:
        mixed_vs_oracle(ring, z, S, 10, K)


@pytest.mark.parametrize("K", [2, st.ST_SPIN_MID_HALF, st.ST_SPIN_MID_KICK])
@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_mixed_drift_kick_ring_against_the_oracle(gg, K):
    """The drift-kick RHIC-like ring (TEAPOT bends, drift-kick quadrupoles and
    sextupoles, snakes), 10 turns, against the oracle."""
    ring = W.with_spin_order(W.drift_kick_ring(W.rhic_like_ring(gg, n_cells=20)), 2)
    z, S = W.gaussian_particles(200, gg, seed=63)
    mixed_vs_oracle(ring, z, S, 10, K)


def test_mixed_drift_kick_ring_with_fringes_and_odd_slices():
    ring = W.with_slices(W.with_fringes(W.drift_kick_ring(W.rhic_like_ring(487.0, n_cells=12))), 3)
    z, S = W.gaussian_particles(200, 487.0, seed=64)
    mixed_vs_oracle(ring, z, S, 10, st.ST_SPIN_MID_KICK)
    ring2 = W.with_spin_order(W.with_fringes(W.drift_kick_ring(W.rhic_like_ring(487.0, n_cells=12))), 2)
    mixed_vs_oracle(ring2, z, S, 10, 2)


@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_mixed_drift_kick_ring_1000_turns_within_1e_6(gg):
    """1000 turns of the full drift-kick RHIC-like ring: the mixed tracker
    against the FP64 tracker (itself at parity with the oracle), mean Delta S
    within 1e-6, orbit within 1e-6."""
    ring = W.with_spin_order(W.drift_kick_ring(W.rhic_like_ring(gg)), 2)
    z, S = W.gaussian_particles(1024, gg, seed=3452)
    zm, Sm, lm = st.track(ring, z, S, 1000, 2, precision="mixed")
    zf, Sf, lf = st.track(ring, z, S, 1000, 2)
    assert np.array_equal(lm, lf)
    mean, mx = spin_err(Sm, Sf)
    dz = np.abs(zm - zf).max(axis=1)
    print(f"TEAPOT ring, G gamma0 = {gg}: mixed vs FP64 after 1000 turns: dS mean {mean:.3e} max {mx:.3e}, "
          f"orbit {dz[:5]}")
    assert mean <= 1e-6, (mean, mx)
    assert dz[:4].max() < 1e-6


def test_mixed_teapot_lost_particles_and_orbit_only():
    """Particles lost in a TEAPOT bend (a line that never meets the turned
    frame; an imaginary Ps) are flagged and keep their entrance state as in the
    oracle; the orbit-only mode tracks the same orbit."""
    gg = 45.5
    ring = W.with_spin_order(W.drift_kick_ring(W.toy_ring(gg)), 2)
    ring["elements"] = [e for e in ring["elements"] if e["type"] == "teapot"][:1] + ring["elements"]
    z, S = W.gaussian_particles(40, gg, seed=4)
    z[1, 5], z[3, 5], z[5, 5] = 0.9995, 0.0, 0.0
    z[3, 21] = -1.2
    zm, Sm, lm = mixed_vs_oracle(ring, z, S, 3, 2)
    assert lm[5] == 1 and lm[21] == 1 and lm.sum() == 2
    # the entrance state, to the 48 bits of the compensated pairs
    assert np.abs(zm[:, 21] - z[:, 21]).max() <= 1e-14 * np.abs(z[:, 21]).max()
    assert np.abs(zm[:, 5] - z[:, 5]).max() <= 1e-14 * np.abs(z[:, 5]).max()
    assert np.array_equal(Sm[:, 5], S[:, 5]) and np.array_equal(Sm[:, 21], S[:, 21])
    lat = st.Lattice(ring)
    tr = st.Tracker(lat, 40, "mixed")
    tr.upload(z, S)
    tr.track_orbit(3)
    zo, So, lo = tr.download()
    tr.close()
    lat.close()
    # the orbit-only kernel may contract FP32 operations differently
    assert np.array_equal(lo, lm) and np.array_equal(So, S)
    alive = lm == 0
    assert np.abs(zo[:4, alive] - zm[:4, alive]).max() < 1e-9
    assert np.array_equal(zo[:, ~alive], zm[:, ~alive])
