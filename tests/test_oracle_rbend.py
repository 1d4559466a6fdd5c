"""Pins of the oracle's rectangular bend (Sec. 3.2: Eqs. (rhob), (rbend),
(Hprot), (prot), (dipolefringe), (Xoffset), (Toffset); Sec. 4.5: Eq.
(skfringeRB)) against facts that do not come from the oracle: Hamilton's
equations of the body and of the dynamic rotation integrated numerically, the
on-axis closed form, an independent lab-frame construction of the whole
magnet for particles in the mid-plane (face planes, a hard-edge field
region, the reference trajectory integrated numerically, the Thomas-BMT
rotation of the spin by (1 + G gamma) times the turn of the velocity),
symplecticity of the thin-fringe map, and the Lorentz force and Thomas-BMT
through a fringe whose field rises linearly over a vanishing length."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
import workloads as W

G = W.G_PROTON
OMEGA6 = np.kron(np.eye(3), np.array([[0.0, 1.0], [-1.0, 0.0]]))


def ref_consts(gg):
    gamma0 = gg / G
    return gamma0, math.sqrt(1 - 1 / gamma0 ** 2)


def P2(pt, beta0):
    return 1 + 2 * pt / beta0 + pt * pt


def states(gg, n=4, seed=2, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        out.append(np.array([3e-3 * rng.standard_normal(), 2e-2 + 3e-4 * rng.standard_normal(),
                             2e-3 * rng.standard_normal(), 3e-4 * rng.standard_normal(),
                             1e-2 * rng.standard_normal(), float(W.delta_to_pt(np.array(1e-3), gg))]) * scale)
    return out


# ---------------------------------------------------------------------------
# body and dynamic rotation against Hamilton's equations
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_body_matches_hamilton_ode(gg):
    """Eq. (rbend) against H = -Ps + b X (the printed T excludes the 1/beta0
    term, which Eq. (Toffset) accounts for)."""
    _, beta0 = ref_consts(gg)
    b = 0.03
    for z in states(gg):
        def f(_, y):
            Ps = math.sqrt(P2(y[5], beta0) - y[1] ** 2 - y[3] ** 2)
            return [y[1] / Ps, -b, y[3] / Ps, 0.0, -(1 / beta0 + y[5]) / Ps, 0.0]
        ref = solve_ivp(f, (0, 2.0), z, method="DOP853", rtol=1e-13, atol=1e-16).y[:, -1]
        out, rc = oracle.subflow("rbend_body", G, gg, z, 2.0, k1=b)
        assert rc == 0
        assert np.abs(out - ref).max() < 1e-13


@pytest.mark.parametrize("phi", [0.05, -0.3, 0.7])
def test_dynamic_rotation_is_the_flow_of_h_prot(phi):
    """Eq. (prot) against Hamilton's equations of H_prot = -X Ps with phi as
    the independent variable (Eq. (Hprot)), including the sign of the T
    update."""
    gg = 45.5
    _, beta0 = ref_consts(gg)
    for z in states(gg, scale=3.0):
        def f(_, y):
            Ps = math.sqrt(P2(y[5], beta0) - y[1] ** 2 - y[3] ** 2)
            return [y[0] * y[1] / Ps, Ps, y[0] * y[3] / Ps, 0.0, -y[0] * (1 / beta0 + y[5]) / Ps, 0.0]
        ref = solve_ivp(f, (0, phi), z, method="DOP853", rtol=1e-13, atol=1e-16).y[:, -1]
        out, rc = oracle.subflow("rbend_rotation", G, gg, z, phi)
        assert rc == 0
        assert np.abs(out - ref).max() < 1e-14


def _jacobian(fun, z0):
    J = np.zeros((6, 6))
    for j in range(6):
        zc = np.array(z0, dtype=np.complex128)
        zc[j] += 1e-30j
        J[:, j] = fun(zc).imag / 1e-30
    return J


@pytest.mark.parametrize("which,k1,k2,s", [("rbend_fringe", 0.05, 1.0, 0.0), ("rbend_fringe", 0.05, -1.0, 0.0),
                                           ("rbend_rotation", 0.0, 0.0, 0.2), ("rbend_body", 0.03, 0.0, 1.5)])
def test_pieces_are_symplectic(which, k1, k2, s):
    gg = 45.5
    for z0 in states(gg, scale=5.0):
        J = _jacobian(lambda zc: oracle.subflow(which, G, gg, zc, s, k1=k1, k2=k2, variant="c128")[0], z0)
        assert np.abs(J.T @ OMEGA6 @ J - OMEGA6).max() < 1e-12


# ---------------------------------------------------------------------------
# whole element
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("e1", [0.0, 0.01, -0.02])
@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_on_axis_reference_particle(e1, gg):
    """The reference particle leaves on the axis with T = 0, and its spin has
    turned by -G gamma0 * angle about y, as in a sector bend of the same angle."""
    ang = 0.04
    el = W.element("rbend", L=3.0, n_slices=8, angle=ang, e1=e1)
    S0 = np.array([0.0, 0.0, 1.0])
    z, S, _, _, rc = oracle.element_detail(el, G, gg, np.zeros(6), S0, 2)
    assert rc == 0
    assert np.abs(z).max() < 2e-15
    th = -gg * ang
    np.testing.assert_allclose(S, [math.sin(th), 0.0, math.cos(th)], rtol=0, atol=2e-13)


def _lab_frame_rbend(el, gg, z, S):
    """Independent construction for a particle in the mid-plane (Y = Py = 0):
    entrance reference plane z_lab = 0 through the reference point, entrance
    face through the same point with its normal at phi_entr to the
    reference direction, a uniform field b between the faces (hard edges),
    straight lines outside; the reference trajectory is integrated like the
    particle's in the design field (eta = 1), and the exit reference frame is
    its exit point and direction (the magnet's placement does not depend on
    a field error).
    T changes by (reference path)/beta0 - (particle path)/beta; the spin turns
    about y by (1 + G gamma) times the turn of the velocity in the field, and
    its components are taken in each frame."""
    gamma0, beta0 = ref_consts(gg)
    phi_in, phi_out = 0.5 * el["angle"] + el["e1"], -0.5 * el["angle"] + el["e1"]
    L = el["L"]
    b_design = (math.sin(phi_in) - math.sin(phi_out)) / L
    xm = np.array([math.cos(phi_in), math.sin(phi_in)])          # magnet axes in lab (x, z)
    zm = np.array([-math.sin(phi_in), math.cos(phi_in)])

    def to_m(v):
        return np.array([v @ xm, v @ zm])

    def ray(X, Px, Pt, b):
        P = math.sqrt(P2(Pt, beta0))
        Ps = math.sqrt(P * P - Px * Px)
        p = to_m(np.array([X, 0.0]))
        d = to_m(np.array([Px, Ps]) / P)
        t = -p[1] / d[1]                       # to the entrance face z_m = 0
        p = p + t * d
        length = t
        pxm = P * d[0]

        def f(_, y):                           # y = (x_m, Px_m, path) against z_m
            ps = math.sqrt(P * P - y[1] ** 2)
            return [y[1] / ps, -b, P / ps]
        sol = solve_ivp(f, (0.0, L), [p[0], pxm, 0.0], method="DOP853", rtol=1e-13, atol=1e-16).y[:, -1]
        pxf = sol[1]
        df = np.array([pxf, math.sqrt(P * P - pxf * pxf)]) / P
        turn = math.atan2(df[0], df[1]) - math.atan2(d[0], d[1])
        return np.array([sol[0], L]), df, length + sol[2], turn, P

    qref, dref, lref, _, _ = ray(0.0, 0.0, 0.0, b_design)
    ze = dref                                    # exit frame axes (magnet components)
    xe = np.array([dref[1], -dref[0]])
    q, d, length, turn, P = ray(z[0], z[1], z[5], el["eta"] * b_design)
    t = -((q - qref) @ ze) / (d @ ze)            # straight to the exit reference plane
    q = q + t * d
    length += t
    inv_beta = (1 / beta0 + z[5]) / P
    X = (q - qref) @ xe
    Px = P * (d @ xe)
    T = z[4] + lref / beta0 - length * inv_beta

    def roty(a, v):
        return np.array([v[0] * math.cos(a) + v[2] * math.sin(a), v[1], -v[0] * math.sin(a) + v[2] * math.cos(a)])
    gamma = gamma0 * (1 + beta0 * z[5])
    Sm = roty(phi_in, S)                         # components in the magnet frame
    Sm = roty((1 + G * gamma) * turn, Sm)        # Thomas-BMT in a transverse field
    Se = roty(-math.atan2(dref[0], dref[1]), Sm)                        # components in the exit frame
    return np.array([X, Px, 0.0, 0.0, T, z[5]]), Se


@pytest.mark.parametrize("e1", [0.0, 0.015])
@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_mid_plane_particles_match_the_lab_frame_construction(e1, gg):
    ang = 0.08
    el = W.element("rbend", L=3.0, n_slices=64, angle=ang, e1=e1, eta=1.002)
    rng = np.random.default_rng(11)
    for _ in range(4):
        z = np.array([2e-3 * rng.standard_normal(), 4e-4 * rng.standard_normal(), 0.0, 0.0,
                      1e-2 * rng.standard_normal(), float(W.delta_to_pt(np.array(2e-3 * rng.standard_normal()), gg))])
        S0 = rng.standard_normal(3)
        S0 /= np.linalg.norm(S0)
        zo, So, _, _, rc = oracle.element_detail(el, G, gg, z, S0, 3)
        assert rc == 0
        zl, Sl = _lab_frame_rbend(el, gg, z, S0)
        np.testing.assert_allclose(zo, zl, rtol=0, atol=1e-12)
        np.testing.assert_allclose(So, Sl, rtol=0, atol=1e-10)


# ---------------------------------------------------------------------------
# thin fringe: orbit focusing and spin kick against a linear fringe
# ---------------------------------------------------------------------------

def _ramp(z, S, b, eps, sign, gg):
    """Lorentz force (kinetic momenta) and Thomas-BMT in the magnet's frame
    through a fringe of length eps with the field of the potential g(s) b Y:
    (0, g b, g' b Y), g rising (sign +1) or falling (-1) linearly."""
    gamma0, beta0 = ref_consts(gg)
    P = math.sqrt(P2(z[5], beta0))
    gamma = gamma0 * (1 + beta0 * z[5])

    def rhs(s, y):
        X, px, Y, py = y[:4]
        g, gp = (s / eps, 1 / eps) if sign > 0 else (1 - s / eps, -1 / eps)
        bv = np.array([0.0, g * b, gp * b * Y])
        ps = math.sqrt(P * P - px * px - py * py)
        u = np.array([px, py, ps]) / P
        b_par = (u @ bv) * u
        om = -(1 / ps) * ((1 + G * gamma) * (bv - b_par) + (1 + G) * b_par)
        return np.concatenate([[px / ps, (py * bv[2] - ps * bv[1]) / ps, py / ps, (ps * bv[0] - px * bv[2]) / ps],
                               np.cross(om, y[4:])])
    sol = solve_ivp(rhs, (0.0, eps), np.concatenate([z[:4], S]), method="DOP853", rtol=1e-13, atol=1e-17)
    return sol.y[:4, -1], sol.y[4:, -1]


def _rot(w, S):
    th = np.linalg.norm(w)
    n = w / th
    return S * math.cos(th) + np.cross(n, S) * math.sin(th) + n * (n @ S) * (1 - math.cos(th))


@pytest.mark.parametrize("sign", [+1, -1])
def test_fringe_vertical_focusing_is_the_thin_limit_of_a_linear_fringe(sign):
    """A particle crossing the face at x' = Px/Ps receives
    dPy = -(+-b) x' Y (Eq. (vertfocus)) to lowest order; extrapolated to
    eps -> 0 the Lorentz-force result agrees to relative order of the
    amplitudes."""
    gg, b = 45.5, 0.02
    mism = []
    for lam in (1.0, 0.5):
        z = np.array([2e-3, 0.03, 4e-3, 2e-4, 0.0, 0.0]) * lam
        out, rc = oracle.subflow("rbend_fringe", G, gg, z, 0.0, k1=b, k2=float(sign))
        assert rc == 0
        dpy = [(_ramp(z, np.array([0.0, 0.0, 1.0]), b, eps, sign, gg)[0][3] - z[3]) for eps in (2e-5, 1e-5)]
        dpy0 = 2 * dpy[1] - dpy[0]
        kick = out[3] - z[3]
        assert abs(kick) > 1e-7
        mism.append(abs(dpy0 - kick) / abs(kick))
    assert mism[0] < 1e-2 and mism[1] < 0.6 * mism[0], mism


@pytest.mark.parametrize("sign", [+1, -1])
def test_fringe_spin_kick_is_the_thin_limit_of_a_linear_fringe(sign):
    """Eq. (skfringeRB) (read with its factor Y): a particle crossing at a
    large horizontal angle sees part of the longitudinal fringe field
    transverse to its velocity.  The x and s components of the kick agree with
    the extrapolated Thomas-BMT rotation to relative order of the amplitudes
    at G gamma = 487, where the x component is the larger one."""
    gg = 487.0
    el = W.element("rbend", L=2.0, n_slices=8, angle=0.04, fringe=1)
    S0 = np.array([0.0, 1.0, 0.0])
    ratios = []
    for lam in (1.0, 0.5):
        z = np.array([1e-3, 0.04 * lam, 3e-3 * lam, 1e-4 * lam, 0.0, 0.0])
        bs = el["eta"] * (math.sin(0.02) - math.sin(-0.02)) / el["L"]
        w, rc = oracle.element_fringe(el, sign, G, gg, z)
        assert rc == 0
        Ss = [_ramp(z, S0, bs, eps, sign, gg)[1] for eps in (2e-5, 1e-5)]
        S_ode = 2 * Ss[1] - Ss[0]
        S_kick = _rot(w, S0)
        assert abs(w[0]) > 2 * abs(w[2])
        ratios.append(np.abs(S_ode - S_kick).max() / np.linalg.norm(w))
    assert ratios[0] < 0.05 and ratios[1] < 0.6 * ratios[0], ratios


def test_rbend_validation():
    for el in (W.element("rbend", L=2.0, n_slices=4, angle=0.0),
               W.element("rbend", L=2.0, n_slices=4, angle=0.1, eta=0.0),
               W.element("rbend", L=2.0, n_slices=4, angle=0.1, e1=1.6)):
        assert not oracle.check_lattice(W.single_element_ring(el, 45.5), 0)
    assert oracle.check_lattice(W.single_element_ring(W.element("rbend", L=2.0, n_slices=4, angle=0.1), 45.5), 2)
