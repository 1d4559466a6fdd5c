"""Pins of the oracle's thin lens (Sec. 3.5: the multipole of Sec. 3.4 in the
limit of zero length at fixed integrated strengths) against facts that do not
come from the oracle: the flow of the multipole potential over a unit kick
parameter (sympy-differentiated, tests/ode_reference.py), and Hamilton's
equations with the Thomas-BMT equation integrated numerically through a
thick multipole of length eps -> 0 at the same integrated strengths."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from ode_reference import integrate

G = W.G_PROTON
S0 = np.array([0.3, 0.2, math.sqrt(1 - 0.13)])
K1L, K2L = 0.05, 1.5


def z_start(gg):
    return np.array([4e-3, 3e-4, -3e-3, 2e-4, 1e-3, float(W.delta_to_pt(np.array(2e-3), gg))])


@pytest.mark.parametrize("N", [1, 2, 8])
def test_thin_lens_orbit_is_the_flow_of_the_multipole_potential(N):
    """Positions, T and Pt unchanged; (Px, Py) kicked by the field of the
    integrated strengths whatever the slicing (the partial kicks commute)."""
    gg = 45.5
    z0 = z_start(gg)
    zo, rc = oracle.orbit_map(W.element("thin_mult", n_slices=N, k1=K1L, k2=K2L), G, gg, z0)
    assert rc == 0
    zr = integrate("kick", z0, 1.0, G, gg, k1=K1L, k2=K2L)
    assert np.abs(zo - zr).max() < 1e-17
    assert np.array_equal(zo[[0, 2, 4, 5]], z0[[0, 2, 4, 5]])


@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_thin_lens_is_the_zero_length_limit_of_the_thick_multipole(gg):
    """Against Hamilton's and Thomas-BMT's equations through a thick
    multipole of length eps with strengths K1L/eps, K2L/eps: the difference
    falls in proportion to eps (the thick element's drift over eps), and the
    limit extrapolated from eps = 1e-4 and 1e-5 agrees with the thin lens
    (64 slices, three Romberg steps) to 1e-13."""
    z0 = z_start(gg)
    _, S, _, _, rc = oracle.element_detail(W.element("thin_mult", n_slices=64, k1=K1L, k2=K2L), G, gg, z0, S0, 3)
    assert rc == 0
    Ss = [integrate("mult", z0, eps, G, gg, k1=K1L / eps, k2=K2L / eps, S0=S0, rtol=1e-13, atol=1e-18)[1]
          for eps in (1e-4, 1e-5)]
    d = [np.abs(S - Sr).max() for Sr in Ss]
    assert 9.0 < d[0] / d[1] < 11.0, d
    assert np.abs(S - (Ss[1] + (Ss[1] - Ss[0]) / 9.0)).max() < 1e-13
    # the rotation is not small: the thin lens turns the spin
    assert np.abs(S - S0).max() > 1e-3 * (gg / 45.5)


def test_thin_lens_spin_converges_at_the_romberg_rates():
    """Refining the sampling of the kick: the trapezoid levels converge as
    N^-2 and one Romberg step as N^-4 towards the 256-slice, three-step
    result."""
    gg = 487.0
    z0 = z_start(gg) * 3.0
    z0[5] = float(W.delta_to_pt(np.array(2e-3), gg))
    el = lambda N: W.element("thin_mult", n_slices=N, k1=0.3, k2=8.0)
    _, Sref, _, _, _ = oracle.element_detail(el(256), G, gg, z0, S0, 3)
    for K, lo, hi in ((0, 3.6, 4.4), (1, 13.0, 19.0)):
        e = []
        for N in (4, 8, 16):
            _, S, _, _, _ = oracle.element_detail(el(N), G, gg, z0, S0, K)
            e.append(np.linalg.norm(S - Sref))
        assert all(lo < e[i] / e[i + 1] < hi for i in range(2)), (K, e)


def test_ring_with_thin_sextupoles_matches_thick_ones_closely():
    """The RHIC-like ring with its 0.2 m sextupoles replaced by thin lenses of
    the same integrated strength between half drifts tracks close to the
    thick-sextupole ring (the two differ by the sextupoles' finite length)."""
    gg = 45.5
    ring = W.rhic_like_ring(gg, n_cells=12)
    thin = W.with_thin_sextupoles(ring)
    assert len(thin["elements"]) == len(ring["elements"]) + 2 * 24
    z, S = W.gaussian_particles(16, gg, seed=2)
    z1, S1, l1 = oracle.track(ring, z, S, 1, 1)
    z2, S2, l2 = oracle.track(thin, z, S, 1, 1)
    assert not l1.any() and not l2.any()
    assert 0.0 < np.abs(z1 - z2)[:4].max() < 1e-5 and np.abs(S1 - S2).max() < 1e-5


def test_thin_lens_validation():
    ok = W.single_element_ring(W.element("thin_mult", n_slices=4, k2=1.0), 45.5)
    assert oracle.check_lattice(ok, 2) and oracle.check_lattice(ok, oracle.MID_KICK)
    for el in (W.element("thin_mult", L=0.1, n_slices=4, k2=1.0),
               W.element("thin_mult", n_slices=4, k2=1.0, fringe=1),
               W.element("thin_mult", n_slices=4, k2=1.0, split_order=4),
               W.element("thin_mult", n_slices=3, k2=1.0)):
        assert not oracle.check_lattice(W.single_element_ring(el, 45.5), 2)
