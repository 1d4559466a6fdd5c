"""The paper's statements about orbital errors (Sec. 5.1, Figs. oneTurnErrsX
and xErrVsTurnNo) as checks on a tracker, `track(ring, z, S, n_turns,
spin_order)` returning (z, S, lost): the oracle or the CUDA library.  The
reference runs are the oracle's.  The ring is the RHIC-scale ring with thin
sextupoles (Sec. 3.5), whose thin kicks are exact at any slicing, so the
bend-kick / matrix-kick errors are those of the matrix-kick split alone;
its drift-kick version has TEAPOT bends and drift-kick-drift quadrupoles."""
from __future__ import annotations

import numpy as np

import oracle
import workloads as W

GG = 45.5


def rings():
    base = W.with_thin_sextupoles(W.rhic_like_ring(GG))
    return base, W.drift_kick_ring(base)


def relative_dX(zx, zref):
    """Delta X of Sec. 5.1 (rms over the bunch of X - X_ref) relative to the
    rms of X_ref."""
    return float(np.sqrt(np.mean((zx[0] - zref[0]) ** 2)) / np.sqrt(np.mean(zref[0] ** 2)))


def check_one_turn_errors(track, n_particles=64):
    """Fig. oneTurnErrsX: one-turn Delta X(1; n_b) against bend-kick /
    matrix-kick with n_b = 128.  Both integrators converge as n_b^-2; drift-kick
    starts at a relative error of order one and reaches about a part in 1e4 at
    n_b = 64; bend-kick / matrix-kick starts below a part in 1e6 and falls
    below a part in 1e9."""
    base, dk = rings()
    z, S = W.gaussian_particles(n_particles, GG, seed=9)
    zr, _, lr = oracle.track(W.with_slices(base, 128), z, S, 1, 0)
    assert not lr.any()
    err = {}
    for name, ring in (("dk", dk), ("bk", base)):
        for nb in (1, 2, 4, 8, 16, 32, 64):
            z1, _, l1 = track(W.with_slices(ring, nb), z, S, 1, 0)
            assert not l1.any()
            err[(name, nb)] = relative_dX(z1, zr)
    assert err[("dk", 1)] > 0.1
    assert 0.5e-4 < err[("dk", 64)] < 5e-4
    assert all(3.5 < err[("dk", nb)] / err[("dk", 2 * nb)] < 4.5 for nb in (4, 8, 16, 32))
    assert err[("bk", 1)] < 1e-6
    assert min(err[("bk", nb)] for nb in (32, 64)) < 1e-9
    assert all(3.3 < err[("bk", nb)] / err[("bk", 2 * nb)] < 4.5 for nb in (2, 4, 8))
    return err


def check_errors_over_turns(track, turns=30, n_particles=64):
    """Fig. xErrVsTurnNo, against bend-kick / matrix-kick with n_b = 16: at
    every turn drift-kick with n_b = 8 (no tune fit) lies far above
    bend-kick / matrix-kick with n_b = 1, which lies above n_b = 4; the
    drift-kick error oscillates (it falls again at some turns) because of its
    tune error."""
    base, dk = rings()
    z, S = W.gaussian_particles(n_particles, GG, seed=9)
    ref = W.with_slices(base, 16)
    runs = {"dk8": W.with_slices(dk, 8), "bk1": W.with_slices(base, 1), "bk4": W.with_slices(base, 4)}
    state = {k: z for k in runs}
    zr = z
    hist = []
    for _ in range(turns):
        zr, _, _ = oracle.track(ref, zr, S, 1, 0)
        row = {}
        for k, ring in runs.items():
            state[k], _, lk = track(ring, state[k], S, 1, 0)
            assert not lk.any()
            row[k] = relative_dX(state[k], zr)
        assert row["dk8"] > 1e3 * row["bk1"] > 1e3 * row["bk4"], row
        hist.append(row["dk8"])
    assert any(hist[i + 1] < hist[i] for i in range(turns - 1))
    return hist


def check_amplitude_dependence(track, n_particles=400, bin_size=80):
    """Fig. xErrVsAmp: one-turn errors in X binned by amplitude
    (X^2 + (20 m Px)^2, bins of equal count) for drift-kick with n_b = 32
    (upper curve) and bend-kick / matrix-kick with n_b = 1 (lower curve):
    the drift-kick error lies more than 1e3 times above in every bin, and
    the two have roughly the same amplitude dependence (their ratio varies
    by less than a factor 5 across the bins)."""
    base, dk = rings()
    z, S = W.gaussian_particles(n_particles, GG, seed=13)
    zr, _, _ = oracle.track(W.with_slices(base, 128), z, S, 1, 0)
    zd, _, ld = track(W.with_slices(dk, 32), z, S, 1, 0)
    zb, _, lb = track(W.with_slices(base, 1), z, S, 1, 0)
    assert not ld.any() and not lb.any()
    order = np.argsort(z[0] ** 2 + (20.0 * z[1]) ** 2)
    ratios = []
    for b in range(0, n_particles, bin_size):
        idx = order[b:b + bin_size]
        ed = np.sqrt(np.mean((zd[0, idx] - zr[0, idx]) ** 2))
        eb = np.sqrt(np.mean((zb[0, idx] - zr[0, idx]) ** 2))
        assert ed > 1e3 * eb, (b, ed, eb)
        ratios.append(ed / eb)
    assert max(ratios) < 5.0 * min(ratios), ratios
    return ratios


def linear_tunes(J):
    """Fractional horizontal and vertical tunes from the 2x2 diagonal blocks of
    a one-turn Jacobian (uncoupled, stable motion)."""
    import math
    return [math.acos(0.5 * np.trace(J[i:i + 2, i:i + 2])) / (2.0 * math.pi) for i in (0, 2)]


def check_tunes(jacobian, tol_bk):
    """Sec. 5.1 (orbital spectra and tunes; drift-kick needs a tune fit): on
    the RHIC-scale ring with thin sextupoles and no snakes, the bend-kick /
    matrix-kick one-turn linear map is exact at any slice count (exact
    sector-bend map, exact linear quadrupole flow), so its tunes do not move
    with n_b; the drift-kick tunes are off at few slices and converge to them
    as n_b^-2.  jacobian(ring) returns the 6x6 one-turn Jacobian at z = 0."""
    base = W.with_thin_sextupoles(W.rhic_like_ring(GG, snakes=False))
    dk = W.drift_kick_ring(base)
    bk = [linear_tunes(jacobian(W.with_slices(base, nb))) for nb in (1, 4, 16)]
    for t in bk[1:]:
        assert max(abs(a - b) for a, b in zip(t, bk[0])) < tol_bk, (bk, tol_bk)
    d = [max(abs(a - b) for a, b in zip(linear_tunes(jacobian(W.with_slices(dk, nb))), bk[0])) for nb in (4, 16)]
    assert d[0] > 1e-3 and 13.0 < d[0] / d[1] < 19.0, d
    return bk[0], d
