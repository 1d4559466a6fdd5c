"""The paper's statements about its single-element error maps (Sec. 5.2.1),
as checks on a tracker: `track(ring, z, S, n_turns, spin_order)` returning
(z, S, lost), the oracle or the CUDA library.  The reference solution is
always the oracle's, as in the paper's own studies a finely sliced run with
Romberg iterations."""
from __future__ import annotations

import numpy as np

import oracle
import paper_studies as P


def check_dipole_maps(track, Py, Pt):
    """Figs. sbendErrsQ/R and sbendErrsQR4M/QR8M, RHIC dipole, X +-5 cm, Px
    +-6 mrad, reference 128 slices + one Romberg step:
    - piece-wise constant (PWC) errors span the maps' grey scale, below 1e-7.5;
    - one Romberg step lowers the error at every point for 4 and 8 slices
      (except where both are at the rounding level, below 1e-15);
    - the valley of the PWC error follows the locus of Eq. (dpx0): in every
      row of fixed X whose locus lies inside the window, the Px of the
      smallest error is within one grid step of Px_sym(X).
    Returns the error maps {(N, K): [nx, npx]}."""
    z, S, X, PX = P.dipole_grid(Py, Pt)
    _, Sref, lref = oracle.track(P.dipole(128), z, S, 1, 1)
    assert not lref.any()
    maps = {}
    for N in (4, 8):
        for K in (0, 1):
            _, S1, l1 = track(P.dipole(N), z, S, 1, K)
            assert not l1.any()
            maps[(N, K)] = np.linalg.norm(S1 - Sref, axis=0).reshape(len(X), len(PX))
    for N in (4, 8):
        pwc, rom = maps[(N, 0)], maps[(N, 1)]
        assert pwc.max() < 10 ** -7.5, (N, pwc.max())
        assert np.all((rom < pwc) | (np.maximum(rom, pwc) < 1e-15)), N
    step = PX[1] - PX[0]
    sym = P.px_sym(X, Py, Pt)
    inside = np.isfinite(sym) & (sym > PX[0] + step) & (sym < PX[-1] - step)
    valley = PX[np.argmin(maps[(4, 0)], axis=1)]
    assert inside.sum() >= 5
    assert np.abs(valley - sym)[inside].max() <= step, (valley, sym)
    return maps


def check_quad_maps(track, alpha_deg):
    """Fig. quadErrs48QR, RHIC IR quadrupole, X, Y in +-20 mm, spins on a cap
    of half-angle alpha about the vertical, reference 128 slices + three
    Romberg steps; rows 4 and 8 slices PWC, 4 slices + 2 steps, 8 slices + 3
    steps:
    - PWC errors in the maps' range 1e-6 .. 1e-2 (median), falling as N^-2;
    - with two Romberg steps the median error is within 1e-10 .. 10^-5.5, and
      with three steps on 8 slices within 1e-14 .. 10^-8.5;
    - the Romberg maps lie below both PWC maps at every point but the on-axis
      one (no precession at all), and 8 slices + 3 steps below 4 slices + 2
      steps at 95% of the points or more;
    - a vertical spin (alpha = 0): no error in the mid-plane Y = 0, little
      variation with X along a row of fixed Y, growth with |Y| (the field
      (b2 Y, b2 X) is vertical in the mid-plane).
    Returns the error maps {(N, K): [n_points]}."""
    z, S, npt, ms = P.quad_grid(alpha_deg)
    _, Sref, lref = oracle.track(P.ir_quad(128), z, S, 1, 3)
    assert not lref.any()
    maps = {}
    for N, K in ((4, 0), (8, 0), (4, 2), (8, 3)):
        _, S1, l1 = track(P.ir_quad(N), z, S, 1, K)
        assert not l1.any()
        maps[(N, K)] = P.spin_error_map(S1, Sref, npt, ms)
    n = int(round(npt ** 0.5))
    axis = (n // 2) * n + n // 2                       # the on-axis grid point
    off = np.ones(npt, bool)
    off[axis] = False
    for N in (4, 8):
        med = np.median(maps[(N, 0)])
        assert 1e-6 < med < 1e-2 and maps[(N, 0)].max() < 1e-2, (N, med)
    assert 3.7 < np.median(maps[(4, 0)]) / np.median(maps[(8, 0)]) < 4.3
    assert 1e-10 < np.median(maps[(4, 2)]) < 10 ** -5.5
    assert 1e-14 < np.median(maps[(8, 3)]) < 10 ** -8.5
    lo = np.minimum(maps[(4, 0)], maps[(8, 0)])
    if alpha_deg == 0:
        grid = maps[(4, 0)].reshape(n, n)             # [X index, Y index]
        mid = n // 2
        assert grid[:, mid].max() < 1e-15
        rows = [grid[:, j] for j in range(n) if j != mid]
        assert all(r.max() < 1.6 * r.min() for r in rows[:2] + rows[-2:])
        edge = [grid[:, j].mean() for j in range(mid, n)]
        assert all(edge[i] < edge[i + 1] for i in range(len(edge) - 1))
        off &= np.abs(z[2, :npt]) > 0.0             # the mid-plane has no error to lower
    for key in ((4, 2), (8, 3)):
        assert np.all(maps[key][off] < lo[off]), key
    assert np.mean(maps[(8, 3)][off] < maps[(4, 2)][off]) >= 0.95
    return maps
