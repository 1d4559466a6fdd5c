"""Pins of the oracle's thin dipole and multipole fringe spin kicks (Sec. 4.5,
Eq. (skfringe)) against facts that do not come from the oracle: the
Thomas-BMT equation and the Lorentz force integrated numerically through a
fringe whose field rises (entrance) or falls (exit) linearly over a length
eps, with the field of the scalar potential g(s) sum_m (b_m/m) Im (X + iY)^m
(transverse part g times the body field, longitudinal part g' times the sum),
extrapolated to eps -> 0; and whole elements with such fringes at both ends
around the numerically integrated body."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
import workloads as W
from ode_reference import integrate as body_ode

G = W.G_PROTON
S0 = np.array([0.3, 0.2, math.sqrt(1 - 0.13)])


def normal_multipoles(el):
    """(m, b_m/(B rho)) of an element, normalised as in Eq. (Amult)."""
    if el["type"] == "sbend":
        return [(1, el["eta"] * el["angle"] / el["L"])]
    if el["type"] == "quad_mk":
        return [(2, el["k1"])]
    return [(2, el["k1"]), (3, 0.5 * el["k2"])]


def fringe_field(el, X, Y, g, gp):
    """b = B/(B rho) = grad of g(s) Im F(X + iY), F = sum_m (b_m/m) w^m:
    (g Im F', g Re F', g' Im F)."""
    w = complex(X, Y)
    F = Fp = 0j
    for m, b in normal_multipoles(el):
        F += b / m * w ** m
        Fp += b * w ** (m - 1)
    return np.array([g * Fp.imag, g * Fp.real, gp * F.imag])


def ramp(el, z, S, eps, sign, gg):
    """Orbit (kinetic momenta, Lorentz force) and Thomas-BMT spin through a
    straight fringe of length eps whose profile g rises 0 -> 1 (sign +1) or
    falls 1 -> 0 (sign -1).  Returns (z6, S3)."""
    gamma0 = gg / G
    beta0 = math.sqrt(1 - 1 / gamma0 ** 2)
    P2 = 1 + 2 * z[5] / beta0 + z[5] ** 2
    P = math.sqrt(P2)
    gamma = gamma0 * (1 + beta0 * z[5])

    def rhs(s, y):
        X, px, Y, py = y[:4]
        g, gp = (s / eps, 1 / eps) if sign > 0 else (1 - s / eps, -1 / eps)
        b = fringe_field(el, X, Y, g, gp)
        ps = math.sqrt(P2 - px * px - py * py)
        u = np.array([px, py, ps]) / P
        b_par = np.dot(u, b) * u
        om = -(1 / ps) * ((1 + G * gamma) * (b - b_par) + (1 + G) * b_par)
        dz = [px / ps, (py * b[2] - ps * b[1]) / ps, py / ps, (ps * b[0] - px * b[2]) / ps]
        return np.concatenate([dz, np.cross(om, y[4:])])

    sol = solve_ivp(rhs, (0.0, eps), np.concatenate([z[:4], S]), method="DOP853", rtol=1e-13, atol=1e-17)
    assert sol.success
    z1 = np.array(z, dtype=float)
    z1[:4] = sol.y[:4, -1]
    return z1, sol.y[4:, -1]


def rotate(w, S):
    th = np.linalg.norm(w)
    if th == 0.0:
        return S.copy()
    n = w / th
    return S * math.cos(th) + np.cross(n, S) * math.sin(th) + n * np.dot(n, S) * (1 - math.cos(th))


def state(gg, lam):
    z = np.array([8e-3, 4e-3, -5e-3, 6e-3, 0.0, 0.0]) * lam
    z[5] = float(W.delta_to_pt(np.array(2e-3), gg))
    return z


ELEMENTS = [
    ("quadrupole", W.element("quad_mk", L=1.0, n_slices=64, k1=0.8, fringe=1), 2),
    ("sextupole", W.element("mult", L=0.5, n_slices=64, k2=30.0, fringe=1), 3),
    ("quad+sextupole", W.element("mult", L=1.0, n_slices=64, k1=-0.5, k2=20.0, fringe=1), 2),
    ("sector dipole", W.element("sbend", L=2.0, n_slices=64, angle=0.2, fringe=1), 1),
]


@pytest.mark.parametrize("sign", [+1, -1])
@pytest.mark.parametrize("name,el,m", ELEMENTS, ids=[e[0] for e in ELEMENTS])
def test_kick_is_the_thin_limit_of_a_linear_fringe(name, el, m, sign):
    """Extrapolated to eps -> 0, the spin after a linear fringe agrees with the
    rotation of Eq. (skfringe) to relative order of the transverse amplitudes
    (the formula is the lowest order in the dynamical variables): at
    amplitudes of 1e-2 the mismatch is below 2e-3 of the kick, and halving
    every amplitude divides it by at least 0.75 * 2^(m+1)."""
    gg = 2.5
    mism, kick = [], []
    for lam in (1.0, 0.5):
        z = state(gg, lam)
        w, rc = oracle.element_fringe(el, sign, G, gg, z)
        assert rc == 0
        assert w[0] == 0.0 and w[1] == 0.0
        Ss = [ramp(el, z, S0, eps, sign, gg)[1] for eps in (2e-5, 1e-5)]
        mism.append(np.abs(2 * Ss[1] - Ss[0] - rotate(w, S0)).max())
        kick.append(abs(w[2]))
    assert kick[0] > 1e-6
    assert mism[0] < 2e-3 * kick[0], (mism, kick)
    assert mism[0] / mism[1] > 0.75 * 2 ** (m + 1), mism


def test_entrance_and_exit_kicks_cancel_for_an_unchanged_orbit():
    """A rising and a falling fringe at the same transverse position are
    opposite rotations about the same axis (Eq. (skfringe) with the sign)."""
    gg = 45.5
    for _, el, _ in ELEMENTS:
        z = state(gg, 1.0)
        wi, _ = oracle.element_fringe(el, +1, G, gg, z)
        wo, _ = oracle.element_fringe(el, -1, G, gg, z)
        np.testing.assert_array_equal(wi, -wo)


@pytest.mark.parametrize("name,el,m", ELEMENTS, ids=[e[0] for e in ELEMENTS])
def test_element_with_fringes_matches_fringe_body_fringe_ode(name, el, m):
    """Whole element with its fringe flag set (entrance kick, body with 64
    slices and three Romberg iterations, exit kick) against the ODE through
    an entrance ramp, the body (Hamilton's equations and Thomas-BMT), and an
    exit ramp, extrapolated to eps -> 0.  The same element without fringe
    kicks misses the ODE by far more."""
    gg = 2.5
    z = state(gg, 1.0)
    kind = {"quad_mk": "quad", "mult": "mult", "sbend": "sbend"}[el["type"]]
    kw = dict(k1=el["k1"], k2=el["k2"])
    if kind == "sbend":
        kw = dict(h=el["angle"] / el["L"], eta=el["eta"])
    Ss = []
    for eps in (2e-5, 1e-5):
        z1, S1 = ramp(el, z, S0, eps, +1, gg)
        z2, S2 = body_ode(kind, z1, el["L"], G, gg, S0=S1, **kw)
        _, S3 = ramp(el, z2, S2, eps, -1, gg)
        Ss.append(S3)
    S_ode = 2 * Ss[1] - Ss[0]
    _, S_orc, _, _, rc = oracle.element_detail(el, G, gg, z, S0, 3)
    assert rc == 0
    _, S_plain, _, _, _ = oracle.element_detail(dict(el, fringe=0), G, gg, z, S0, 3)
    w_in, _ = oracle.element_fringe(el, +1, G, gg, z)
    err = np.abs(S_orc - S_ode).max()
    assert err < 4e-3 * abs(w_in[2]) + 1e-11, err
    assert np.abs(S_plain - S_ode).max() > 50 * err


def test_fringe_flag_validation():
    ring = W.single_element_ring(W.element("drift", L=1.0, fringe=1), 45.5)
    assert not oracle.check_lattice(ring, 0)
    ring = W.single_element_ring(W.element("mult", L=1.0, n_slices=4, k1=0.1, fringe=2), 45.5)
    assert not oracle.check_lattice(ring, 0)
    ring = W.single_element_ring(W.element("mult", L=1.0, n_slices=4, k1=0.1, fringe=1), 45.5)
    assert oracle.check_lattice(ring, 2)
