"""Pins of the oracle's fourth-order slice map (Sec. 3.3: higher-order
versions of the symmetric split of Eq. (27), here Yoshida's composition of
the second-order map) against facts that do not come from the oracle:
Hamilton's equations integrated numerically (order of convergence), exact
complex-step Jacobians (symplecticity), time reversal, and the Thomas-BMT
equation integrated along the exact orbit (the spin inherits the orbit's
order)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from ode_reference import integrate

G = W.G_PROTON
OMEGA6 = np.kron(np.eye(3), np.array([[0.0, 1.0], [-1.0, 0.0]]))
S0 = np.array([0.3, 0.2, math.sqrt(1 - 0.13)])


def z_start(gg):
    return np.array([3e-3, 3e-4, -2e-3, 2e-4, 0.0, float(W.delta_to_pt(np.array(2e-3), gg))])


CASES = [
    ("mult", dict(type="mult", k1=0.05, k2=0.5), dict(k1=0.05, k2=0.5)),
    ("mult", dict(type="mult", k1=0.5, k2=5.0), dict(k1=0.5, k2=5.0)),
    ("quad", dict(type="quad_mk", k1=-0.5), dict(k1=-0.5)),
]


@pytest.mark.parametrize("kind,el_kw,ode_kw", CASES, ids=["dkd_weak", "dkd_strong", "mk_defocusing"])
def test_orbit_converges_at_fourth_order(kind, el_kw, ode_kw):
    """Halving the slice length divides the orbit error by about 16 with
    split_order 4 (by about 4 with the second-order split of Eq. (27))."""
    gg = 45.5
    z0 = z_start(gg)
    zr = integrate(kind, z0, 1.0, G, gg, **ode_kw)
    for order, lo, hi in ((4, 13.0, 19.5), (2, 3.5, 4.5)):
        errs = []
        for N in (1, 2, 4, 8):
            zo, rc = oracle.orbit_map(W.element(L=1.0, n_slices=N, split_order=order, **el_kw), G, gg, z0)
            assert rc == 0
            errs.append(np.abs(zo - zr)[:4].max())
        ratios = [errs[i] / errs[i + 1] for i in range(3)]
        assert all(lo < r < hi for r in ratios), (order, errs, ratios)


@pytest.mark.parametrize("el", [
    W.element("mult", L=0.4, n_slices=2, k1=0.3, k2=2.0, split_order=4),
    W.element("quad_mk", L=0.5, n_slices=2, k1=0.4, split_order=4),
    W.element("quad_mk", L=0.5, n_slices=2, k1=-0.4, split_order=4),
], ids=["dkd", "mk_f", "mk_d"])
def test_fourth_order_map_is_symplectic_and_reversible(el):
    gg = 487.0
    rng = np.random.default_rng(4)
    back = dict(el, L=-el["L"])
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
        assert np.abs(b - z0).max() < 1e-14


def _spin_errors(el_kw, Sref, gg, z0, order, K, Ns=(4, 8, 16, 32)):
    out = []
    for N in Ns:
        el = W.element(L=1.0, n_slices=N, split_order=order, **el_kw)
        _, S, _, _, rc = oracle.element_detail(el, G, gg, z0, S0, K)
        assert rc == 0
        out.append(np.linalg.norm(S - Sref))
    return out


def test_spin_inherits_the_orbit_order_in_a_drift_kick_multipole():
    """Strong DKD multipole: with the second-order split the spin error
    falls only as N^-2 whatever the Romberg order (the orbit error at the
    slice edges dominates); with the fourth-order map it falls as N^-4."""
    gg = 45.5
    z0 = z_start(gg)
    kw = dict(type="mult", k1=0.5, k2=5.0)
    _, Sref = integrate("mult", z0, 1.0, G, gg, k1=0.5, k2=5.0, S0=S0)
    for K in (1, 2):
        e2 = _spin_errors(kw, Sref, gg, z0, 2, K)
        e4 = _spin_errors(kw, Sref, gg, z0, 4, K)
        assert all(3.6 < e2[i] / e2[i + 1] < 4.4 for i in range(3)), e2
        assert all(14.0 < e4[i] / e4[i + 1] < 18.0 for i in range(3)), e4


def test_fourth_order_map_keeps_the_two_step_romberg_rate_in_a_matrix_kick_quad():
    """Strong MK quadrupole, two Romberg iterations: the spin error falls as
    N^-6 (the paper's rate) only while the orbit's N^-2 split error is below
    it; with the fourth-order map the rate holds down to 2e-14."""
    gg = 45.5
    z0 = z_start(gg)
    kw = dict(type="quad_mk", k1=0.5)
    _, Sref = integrate("quad", z0, 1.0, G, gg, k1=0.5, S0=S0)
    e2 = _spin_errors(kw, Sref, gg, z0, 2, 2)
    e4 = _spin_errors(kw, Sref, gg, z0, 4, 2)
    assert e2[2] / e2[3] < 8.0, e2                     # stalled at the orbit's error
    assert all(45.0 < e4[i] / e4[i + 1] < 90.0 for i in range(1, 3)), e4
    assert e4[3] < 1e-13


def test_split_order_validation():
    for el in (W.element("sbend", L=1.0, n_slices=2, angle=0.1, split_order=4),
               W.element("solenoid", L=1.0, n_slices=2, k1=0.1, split_order=4),
               W.element("mult", L=1.0, n_slices=2, k1=0.1, split_order=3)):
        assert not oracle.check_lattice(W.single_element_ring(el, 45.5), 0)
    assert oracle.check_lattice(W.single_element_ring(W.element("quad_mk", L=1.0, n_slices=2, k1=0.1,
                                                                split_order=4), 45.5), 1)
