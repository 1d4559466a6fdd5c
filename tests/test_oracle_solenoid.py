"""Pins of the oracle's solenoid (Sec. 3.7 body, Sec. 4.4 fringe) against
facts that do not come from the oracle: Hamilton's equations of the solenoid
Hamiltonian integrated numerically (sympy derivatives, DOP853), symplecticity
of the complex-step Jacobian, the on-axis closed form of the spin rotation,
the Thomas-BMT equation integrated through a linear fringe of shrinking
length (the thin-pancake limit), and the convergence statements of the
paper's single-element study (Sec. 5.2.1)."""
import functools
import math

import numpy as np
import pytest
import sympy as sp
from scipy.integrate import solve_ivp

import oracle
import workloads as W

G = W.G_PROTON
M_P = 0.93827208816          # proton mass, GeV
C_LIGHT = 0.299792458        # B rho [T m] = p [GeV/c] / C_LIGHT

X, Px, Y, Py, T, Pt = sp.symbols("X Px Y Py T Pt", real=True)
VARS = (X, Px, Y, Py, T, Pt)
b0s, ks_s, f_s = sp.symbols("beta0 ks f", real=True)


@functools.lru_cache(maxsize=None)
def _solenoid_rhs():
    """Hamilton's equations of -sqrt(P^2 - (Px - Ax)^2 - (Py - Ay)^2) + Pt/beta0
    with the scaled vector potential (Ax, Ay) = f ks/2 (-Y, X) (Eq. (Asol) times
    the fringe profile f)."""
    P2 = 1 + 2 * Pt / b0s + Pt ** 2
    Ax, Ay = -f_s * ks_s / 2 * Y, f_s * ks_s / 2 * X
    H = -sp.sqrt(P2 - (Px - Ax) ** 2 - (Py - Ay) ** 2) + Pt / b0s
    rhs = [sp.diff(H, Px), -sp.diff(H, X), sp.diff(H, Py), -sp.diff(H, Y), sp.diff(H, Pt), -sp.diff(H, T)]
    return sp.lambdify((VARS, b0s, ks_s, f_s), rhs, "numpy")


def _ref(gg):
    gamma0 = gg / G
    return gamma0, math.sqrt(1 - 1 / gamma0 ** 2)


def _precession(z, ks, f, fp, G_, gamma0, beta0):
    """Thomas-BMT with s as independent variable, textbook split of the field
    into parts parallel (1 + G) and transverse (1 + G gamma) to the velocity;
    field from the curl of the vector potential: b = (-f' ks/2 X, -f' ks/2 Y, f ks);
    velocity along the kinetic momentum."""
    b = np.array([-fp * ks / 2 * z[0], -fp * ks / 2 * z[2], f * ks])
    P2 = 1 + 2 * z[5] / beta0 + z[5] ** 2
    px = z[1] + f * ks / 2 * z[2]
    py = z[3] - f * ks / 2 * z[0]
    Ps = math.sqrt(P2 - px * px - py * py)
    u = np.array([px, py, Ps]) / math.sqrt(P2)
    gamma = gamma0 * (1 + beta0 * z[5])
    bpar = np.dot(u, b) * u
    return -(1.0 / Ps) * ((1 + G_ * gamma) * (b - bpar) + (1 + G_) * bpar)


def integrate(z0, s, ks, gg, S0=None, profile=lambda s: (1.0, 0.0), rtol=1e-13, atol=1e-16):
    gamma0, beta0 = _ref(gg)
    f = _solenoid_rhs()

    def rhs(si, y):
        fv, fp = profile(si)
        dz = np.array(f(tuple(y[:6]), beta0, ks, fv), dtype=float)
        if S0 is None:
            return dz
        om = _precession(y[:6], ks, fv, fp, G, gamma0, beta0)
        return np.concatenate([dz, np.cross(om, y[6:])])

    y0 = np.asarray(z0, float) if S0 is None else np.concatenate([z0, S0])
    sol = solve_ivp(rhs, (0.0, s), y0, method="DOP853", rtol=rtol, atol=atol)
    assert sol.success
    return sol.y[:, -1]


def states(gg, n=5, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        d = 1e-3 * rng.standard_normal()
        out.append(np.array([2e-3 * rng.standard_normal(), 2e-4 * rng.standard_normal(),
                             2e-3 * rng.standard_normal(), 2e-4 * rng.standard_normal(),
                             1e-2 * rng.standard_normal(), float(W.delta_to_pt(np.array(d), gg))]))
    return out


def ggamma_of_momentum(p_gev):
    return G * math.sqrt(p_gev ** 2 + M_P ** 2) / M_P


def ks_of(B_tesla, p_gev):
    return B_tesla / (p_gev / C_LIGHT)


@pytest.mark.parametrize("gg,ks", [(45.5, 0.05), (487.0, 0.3), (2.5, 1.5)])
def test_body_map_matches_hamilton_ode(gg, ks):
    for z in states(gg):
        s = 0.7
        zo, rc = oracle.subflow("solenoid", G, gg, z, s, k1=ks)
        assert rc == 0
        zr = integrate(z, s, ks, gg)
        np.testing.assert_allclose(zo, zr, rtol=0, atol=2e-13)


@pytest.mark.parametrize("ks", [0.4, -1.1])
def test_body_map_symplectic_and_reversible(ks):
    gg = 3.0
    from test_oracle_pins import OMEGA6, jacobian
    for z in states(gg, n=3, seed=8):
        J = jacobian(lambda zc: oracle.subflow("solenoid", G, gg, zc, 0.9, k1=ks, variant="c128")[0], z)
        np.testing.assert_allclose(J.T @ OMEGA6 @ J, OMEGA6, rtol=0, atol=1e-12)
        z1, _ = oracle.subflow("solenoid", G, gg, z, 0.9, k1=ks)
        z2, _ = oracle.subflow("solenoid", G, gg, z1, -0.9, k1=ks)
        np.testing.assert_allclose(z2, z, rtol=0, atol=1e-15)


def test_zero_field_is_a_drift():
    gg = 45.5
    for z in states(gg, n=3):
        a, _ = oracle.subflow("solenoid", G, gg, z, 1.3, k1=0.0)
        b, _ = oracle.subflow("drift", G, gg, z, 1.3)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)


@pytest.mark.parametrize("K,N", [(0, 1), (0, 5), (2, 4), (3, 8)])
def test_on_axis_spin_rotation_closed_form(K, N):
    """On axis and on momentum the velocity is along s, the body field is
    parallel to it, Omega = -(1 + G) ks s^ is constant and the fringe kicks
    vanish: the spin turns about s by -(1 + G) ks L for any slicing and order."""
    p = 200.0
    gg = ggamma_of_momentum(p)
    ks = ks_of(1.3, p)
    L = 2.1
    el = W.element("solenoid", L=L, n_slices=N, k1=ks)
    S0 = np.array([0.6, 0.0, 0.8])
    _, S, _, Q, rc = oracle.element_detail(el, G, gg, np.zeros(6), S0, K)
    phi = -(1 + G) * ks * L
    ref = np.array([S0[0] * math.cos(phi) - S0[1] * math.sin(phi), S0[0] * math.sin(phi) + S0[1] * math.cos(phi),
                    S0[2]])
    np.testing.assert_allclose(S, ref, rtol=0, atol=1e-15)
    # the paper's 200 GeV/c case: of order 10 mrad
    assert 8e-3 < abs(phi) < 13e-3


@pytest.mark.parametrize("sign", [+1, -1])
def test_fringe_is_the_thin_limit_of_a_linear_fringe(sign):
    """Thomas-BMT and the orbit integrated through a fringe whose profile
    rises (entrance) or falls (exit) linearly over a length eps.  The result
    differs from the thin limit at first order in eps (the body field inside
    the fringe); extrapolated to eps -> 0 it agrees with the thin-pancake
    rotation of Eq. (solFringe) up to terms of third order in the transverse
    variables (the formula evaluates the fringe at its middle): halving every
    transverse amplitude divides the mismatch by about 8."""
    gg = 2.5
    ks = 1.2
    S0 = np.array([0.3, 0.2, math.sqrt(1 - 0.13)])
    mism = []
    for lam in (1.0, 0.5):
        z = np.array([8e-3, 4e-3, -5e-3, 6e-3, 0.0, 0.0]) * lam
        z[5] = float(W.delta_to_pt(np.array(2e-3), gg))
        w, rc = oracle.solenoid_fringe(ks, sign, G, gg, z)
        assert rc == 0
        th = np.linalg.norm(w)
        nax = w / th
        Sw = S0 * math.cos(th) + np.cross(nax, S0) * math.sin(th) + nax * np.dot(nax, S0) * (1 - math.cos(th))
        Ss = []
        for eps in (2e-5, 1e-5):
            if sign > 0:
                prof = lambda s, e=eps: (s / e, 1.0 / e)
            else:
                prof = lambda s, e=eps: (1.0 - s / e, -1.0 / e)
            y = integrate(z, eps, ks, gg, S0=S0, profile=prof, rtol=1e-13, atol=1e-16)
            Ss.append(y[6:])
            # canonical momenta unchanged across the fringe
            assert abs(y[1] - z[1]) < 1e-6 and abs(y[3] - z[3]) < 1e-6
        # first order in eps: halving eps halves the raw difference
        r1, r2 = np.abs(Ss[0] - Sw).max(), np.abs(Ss[1] - Sw).max()
        assert 1.8 < r1 / r2 < 2.2
        mism.append(np.abs(2 * Ss[1] - Ss[0] - Sw).max())
        assert th > 5e-3
    assert mism[0] < 5e-8
    assert mism[0] / mism[1] > 6.0, mism


def _solenoid_spin(gg, ks, z, S0, N, K):
    el = W.element("solenoid", L=2.1, n_slices=N, k1=ks)
    _, S, _, _, rc = oracle.element_detail(el, G, gg, z, S0, K)
    assert rc == 0
    return S


def test_convergence_of_the_paper_single_element_study():
    """Sec. 5.2.1: a 1.3 T, 2.1 m solenoid.  For 200 GeV/c protons four slices
    with one or two Romberg iterations reach round-off; at low energy (spin
    rotation of order a radian) piece-wise constant integration converges at
    second order and each Romberg iteration removes decades of error."""
    z = np.array([1e-3, 1e-4, -2e-3, -2e-4, 0.0, 0.0])
    S0 = np.array([0.1952, 0.9759, 0.0976])
    S0 /= np.linalg.norm(S0)
    # high energy
    p = 200.0
    gg, ks = ggamma_of_momentum(p), ks_of(1.3, p)
    best = _solenoid_spin(gg, ks, z, S0, 256, 3)
    for K in (1, 2):
        assert np.abs(_solenoid_spin(gg, ks, z, S0, 4, K) - best).max() < 1e-14
    # low energy, 1.2 GeV kinetic
    p = math.sqrt(1.2 ** 2 + 2 * 1.2 * M_P)
    gg, ks = ggamma_of_momentum(p), ks_of(1.3, p)
    best = _solenoid_spin(gg, ks, z, S0, 256, 3)
    e = {N: np.abs(_solenoid_spin(gg, ks, z, S0, N, 0) - best).max() for N in (8, 16, 32, 64)}
    slope = math.log(e[64] / e[8]) / math.log(8.0)
    assert -2.2 < slope < -1.8, slope
    e42 = np.abs(_solenoid_spin(gg, ks, z, S0, 4, 2) - best).max()
    e83 = np.abs(_solenoid_spin(gg, ks, z, S0, 8, 3) - best).max()
    assert e42 < 1e-2 * e[8] and e83 < 1e-2 * e42


def _low_energy_grid():
    """1.2 GeV kinetic-energy protons through the 1.3 T, 2.1 m solenoid of
    Sec. 5.2.1 on a 21 x 21 grid of (Px, Py) in +-3e-3, X = 1 mm, Y = -1 mm,
    spins vertical."""
    p = math.sqrt(1.2 ** 2 + 2 * 1.2 * M_P)
    g = np.linspace(-3e-3, 3e-3, 21)
    PX, PY = np.meshgrid(g, g)
    n = PX.size
    z = np.zeros((6, n))
    z[0], z[2], z[1], z[3] = 1e-3, -1e-3, PX.ravel(), PY.ravel()
    S = np.tile(np.array([[0.0], [1.0], [0.0]]), (1, n))
    return ggamma_of_momentum(p), ks_of(1.3, p), z, S


def test_error_ranges_of_the_paper_solenoid_study_do_not_overlap():
    """Sec. 5.2.1, low-energy solenoid: over the (Px, Py) plane, the spin
    error ranges of 8 slices without Romberg, 4 slices with two Romberg
    iterations and 8 slices with three do not overlap, each lying below the
    previous one; the stand-in for exact tracking is 128 slices with three
    Romberg iterations (the extended-precision build, so that the finest
    range is not rounding noise)."""
    gg, ks, z, S = _low_energy_grid()

    def run(N, K):
        ring = W.single_element_ring(W.element("solenoid", L=2.1, n_slices=N, k1=ks), gg)
        _, So, lost = oracle.track(ring, z, S, 1, K, variant="f80")
        assert not lost.any()
        return So.astype(np.float64)

    ref = run(128, 3)
    err = {nk: np.linalg.norm(run(*nk) - ref, axis=0) for nk in ((8, 0), (4, 2), (8, 3))}
    assert err[(4, 2)].max() < err[(8, 0)].min()
    assert err[(8, 3)].max() < err[(4, 2)].min()


@pytest.mark.parametrize("gg,ks", [(2.5, 1.3), (45.5, 0.08)])
def test_body_spin_matches_thomas_bmt_ode(gg, ks):
    """The whole element against Thomas-BMT integrated through the body (velocity
    along the kinetic momentum, Eq. (mgVSol)) followed by the exit fringe.  The
    particles start on the axis, where the entrance fringe kick vanishes."""
    rng = np.random.default_rng(5)
    L = 2.1
    el = W.element("solenoid", L=L, n_slices=64, k1=ks)
    for _ in range(3):
        z = np.array([0.0, 3e-3 * rng.standard_normal(), 0.0, 3e-3 * rng.standard_normal(), 0.0,
                      float(W.delta_to_pt(np.array(1e-3 * rng.standard_normal()), gg))])
        S0 = rng.standard_normal(3)
        S0 /= np.linalg.norm(S0)
        w_in, _ = oracle.solenoid_fringe(ks, +1, G, gg, z)
        assert np.abs(w_in).max() == 0.0
        zo, So, _, _, rc = oracle.element_detail(el, G, gg, z, S0, 3)
        y = integrate(z, L, ks, gg, S0=S0)
        np.testing.assert_allclose(zo, y[:6], rtol=0, atol=1e-12)
        w, _ = oracle.solenoid_fringe(ks, -1, G, gg, y[:6])
        th = np.linalg.norm(w)
        n = w / th
        Sb = y[6:]
        Se = Sb * math.cos(th) + np.cross(n, Sb) * math.sin(th) + n * np.dot(n, Sb) * (1 - math.cos(th))
        np.testing.assert_allclose(So, Se, rtol=0, atol=1e-11)
