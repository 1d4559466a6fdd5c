"""Pins of the oracle's TEAPOT sector bend (Sec. 3.6: the drift-kick split
H_T = H_D + H_K of a sector bend, Eqs. (DKsplit), (teapotD)) against facts
that do not come from the oracle: Hamilton's equations of the curved drift
and of the whole sector bend integrated numerically (tests/ode_reference.py,
sympy-differentiated Hamiltonians), exact complex-step Jacobians, time
reversal, and the Thomas-BMT equation integrated along the exact orbit."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from ode_reference import integrate

G = W.G_PROTON
OMEGA6 = np.kron(np.eye(3), np.array([[0.0, 1.0], [-1.0, 0.0]]))
S0 = np.array([0.3, 0.2, math.sqrt(1 - 0.13)])


def z_start(gg, scale=1.0):
    z = np.array([3e-3, 3e-4, -2e-3, 2e-4, 1e-3, 0.0]) * scale
    z[5] = float(W.delta_to_pt(np.array(2e-3), gg))
    return z


@pytest.mark.parametrize("h", [0.01, 0.2, -0.05])
@pytest.mark.parametrize("gg", [2.5, 487.0])
def test_curved_drift_is_the_flow_of_the_drift_hamiltonian(h, gg):
    """Eq. (teapotD) with the reference term s/beta0 in T against Hamilton's
    equations of H_D = -(1 + hX) Ps + Pt/beta0 (the sector-bend Hamiltonian
    without field).  The printed form subtracts 1/h from a number of that
    size, so X carries a rounding of a few ulps of 1/h."""
    tol = 1e-15 + 4e-16 / abs(h)
    rng = np.random.default_rng(11)
    for _ in range(4):
        z0 = z_start(gg) * (1.0 + 2.0 * rng.random(6))
        zf, rc = oracle.subflow("curved_drift", G, gg, z0, 0.7, h=h)
        assert rc == 0
        zr = integrate("sbend", z0, 0.7, G, gg, h=h, eta=0.0)
        assert np.abs(zf - zr).max() < tol, np.abs(zf - zr)


def test_curved_drift_without_the_reference_term_misses_the_ode():
    """The printed Eq. (teapotD) has no s/beta0 in T; the ODE of the
    Hamiltonian with its Pt/beta0 term (Eq. (generalH)) needs it."""
    gg = 2.5
    gamma0 = gg / G
    beta0 = math.sqrt(1 - 1 / gamma0 ** 2)
    z0 = z_start(gg)
    zf, _ = oracle.subflow("curved_drift", G, gg, z0, 0.7, h=0.1)
    zr = integrate("sbend", z0, 0.7, G, gg, h=0.1, eta=0.0)
    assert abs((zf[4] - 0.7 / beta0) - zr[4]) > 0.1


def test_teapot_kick_is_the_flow_of_the_field_term():
    """H_K = (eta/2)(1 + hX)^2 (Eq. (sbendA)) depends on X only: its flow
    changes Px by -s dH_K/dX, the derivative taken numerically here (a
    central difference, exact for a quadratic up to rounding)."""
    gg, h, eta, s = 45.5, 0.08, 1.03, 0.4
    z0 = z_start(gg)
    zf, rc = oracle.subflow("teapot_kick", G, gg, z0, s, h=h, eta=eta)
    assert rc == 0

    def HK(X):
        return 0.5 * eta * (1.0 + h * X) ** 2

    e = 0.1
    dH = (HK(z0[0] + e) - HK(z0[0] - e)) / (2 * e)
    assert abs(zf[1] - (z0[1] - s * dH)) < 2e-15
    assert np.array_equal(np.delete(zf, 1), np.delete(z0, 1))


@pytest.mark.parametrize("N", [1, 3, 8])
def test_zero_field_teapot_element_is_exact_for_any_slicing(N):
    gg = 45.5
    z0 = z_start(gg)
    el = W.element("teapot", L=3.0, n_slices=N, angle=0.2, eta=0.0)
    zo, rc = oracle.orbit_map(el, G, gg, z0)
    assert rc == 0
    zr = integrate("sbend", z0, 3.0, G, gg, h=0.2 / 3.0, eta=0.0)
    assert np.abs(zo - zr).max() < 2e-14


@pytest.mark.parametrize("eta", [1.0, 1.01])
def test_teapot_converges_to_the_sector_bend_at_the_split_order(eta):
    """Halving the slice divides the orbit error against Hamilton's equations
    of the sector bend by about 4 (symmetric split, Eq. (27)) or about 16
    (fourth-order composition)."""
    gg = 45.5
    z0 = z_start(gg)
    zr = integrate("sbend", z0, 3.0, G, gg, h=0.2 / 3.0, eta=eta)
    for order, lo, hi in ((2, 3.8, 4.2), (4, 15.0, 17.5)):
        errs = []
        for N in (2, 4, 8, 16):
            el = W.element("teapot", L=3.0, n_slices=N, angle=0.2, eta=eta, split_order=order)
            zo, rc = oracle.orbit_map(el, G, gg, z0)
            assert rc == 0
            errs.append(np.abs(zo - zr).max())
        ratios = [errs[i] / errs[i + 1] for i in range(3)]
        assert all(lo < r < hi for r in ratios), (order, errs, ratios)


def test_teapot_error_constant_is_larger_than_the_bend_kick_map():
    """Sec. 3.6: at the same slice count the TEAPOT orbit is far less accurate
    than the exact sector-bend map of Eq. (10)."""
    gg = 45.5
    z0 = z_start(gg)
    zr = integrate("sbend", z0, 3.0, G, gg, h=0.2 / 3.0, eta=1.0)
    zt, _ = oracle.orbit_map(W.element("teapot", L=3.0, n_slices=4, angle=0.2), G, gg, z0)
    zb, _ = oracle.orbit_map(W.element("sbend", L=3.0, n_slices=4, angle=0.2), G, gg, z0)
    assert np.abs(zt - zr).max() > 1e8 * np.abs(zb - zr).max()


@pytest.mark.parametrize("order", [2, 4])
def test_teapot_map_is_symplectic_and_reversible(order):
    gg = 487.0
    el = W.element("teapot", L=2.0, n_slices=2, angle=0.15, eta=1.02, split_order=order)
    back = dict(el, L=-el["L"], angle=-el["angle"])
    rng = np.random.default_rng(5)
    for _ in range(4):
        z0 = np.array([5e-3, 5e-4, -5e-3, -5e-4, 1e-2, 1e-3]) * rng.standard_normal(6)
        J = np.zeros((6, 6))
        for j in range(6):
            zc = np.array(z0, dtype=np.complex128)
            zc[j] += 1e-30j
            out, _ = oracle.orbit_map(el, G, gg, zc, variant="c128")
            J[:, j] = out.imag / 1e-30
        assert np.abs(J.T @ OMEGA6 @ J - OMEGA6).max() < 1e-12
        a, _ = oracle.orbit_map(el, G, gg, z0)
        b, _ = oracle.orbit_map(back, G, gg, a)
        # every curved drift rounds X to about an ulp of 1/h (see above)
        n_drifts = 2 * el["n_slices"] * (2 if order == 2 else 6)
        assert np.abs(b - z0).max() < 1e-15 + n_drifts * 2.3e-16 * el["L"] / el["angle"]


def test_teapot_spin_follows_the_orbit_order():
    """Against Thomas-BMT integrated along the exact orbit: two Romberg
    iterations give the exact sector bend's N^-6 but only N^-2 on the TEAPOT
    orbit (its slice-edge states carry the split error); the fourth-order
    composition restores N^-4 or better."""
    gg = 45.5
    z0 = z_start(gg)
    h = 0.2 / 3.0
    _, Sref = integrate("sbend", z0, 3.0, G, gg, h=h, eta=1.0, S0=S0)

    def errs(type_, order, K, Ns):
        out = []
        for N in Ns:
            el = W.element(type_, L=3.0, n_slices=N, angle=0.2, split_order=order)
            _, S, _, _, rc = oracle.element_detail(el, G, gg, z0, S0, K)
            assert rc == 0
            out.append(np.linalg.norm(S - Sref))
        return out

    e2 = errs("teapot", 2, 2, (8, 16, 32))
    assert all(3.6 < e2[i] / e2[i + 1] < 4.4 for i in range(2)), e2
    e4 = errs("teapot", 4, 2, (8, 16, 32))
    assert all(e4[i] / e4[i + 1] > 14.0 for i in range(2)), e4
    eb = errs("sbend", 2, 2, (8, 16))
    assert eb[1] < 1e-3 * e2[1], (eb, e2)


def test_teapot_precession_and_fringe_are_those_of_the_sector_bend():
    gg = 45.5
    z0 = z_start(gg)
    for eta in (1.0, 0.98):
        t = W.element("teapot", L=3.0, n_slices=4, angle=0.2, eta=eta, fringe=1)
        b = W.element("sbend", L=3.0, n_slices=4, angle=0.2, eta=eta, fringe=1)
        assert np.array_equal(oracle.omega(t, G, gg, z0)[0], oracle.omega(b, G, gg, z0)[0])
        for sign in (1, -1):
            assert np.array_equal(oracle.element_fringe(t, sign, G, gg, z0)[0],
                                  oracle.element_fringe(b, sign, G, gg, z0)[0])


def test_teapot_ring_on_axis_rotates_by_2pi_G_gamma():
    """A ring of TEAPOT bends without snakes: the on-axis, on-energy spin
    turns about y by -2 pi G gamma0 per turn up to the split error of the
    design orbit, which vanishes as N^-2 (and is large at few slices: the
    half-slice drift leaves the axis by (1/h)(sec(h ds/2) - 1))."""
    gg = 45.5
    ring = W.drift_kick_ring(W.rhic_like_ring(gg, n_cells=8, snakes=False, k1=0.0, k2=0.0))
    z = np.zeros((6, 1))
    S = np.array([[0.0], [0.0], [1.0]])
    dev = []
    for nb in (4, 8):
        _, S1, _ = oracle.track(W.with_slices(ring, nb), z, S, 1, 2)
        a = math.atan2(S1[0, 0], S1[2, 0])
        want = (-2 * math.pi * gg) % (2 * math.pi)
        dev.append(abs((a - want + math.pi) % (2 * math.pi) - math.pi))
    assert 3.5 < dev[0] / dev[1] < 4.5, dev


def test_teapot_validation():
    ok = W.single_element_ring(W.element("teapot", L=3.0, n_slices=4, angle=0.1, fringe=1, split_order=4), 45.5)
    assert oracle.check_lattice(ok, 2)
    for el in (W.element("teapot", L=3.0, n_slices=4, angle=0.0),
               W.element("teapot", L=3.0, n_slices=3, angle=0.1),
               W.element("teapot", L=0.0, n_slices=4, angle=0.1)):
        assert not oracle.check_lattice(W.single_element_ring(el, 45.5), 2)
    # zero field is allowed (a curved drift)
    assert oracle.check_lattice(W.single_element_ring(W.element("teapot", L=3.0, n_slices=4, angle=0.1, eta=0.0),
                                                      45.5), 2)
