"""Pins of the CPU oracle against facts that do not come from the oracle itself:
Hamilton's equations integrated numerically, the Thomas-BMT ODE, closed forms
printed or implied by the paper, textbook matrices, exact invariants, complex-
step Jacobians (symplecticity), time reversibility, and the convergence rates
and single-element results the paper reports (Sec. 5.2.1)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from ode_reference import integrate, precession

G = W.G_PROTON
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def pt_of(delta, gg):
    return float(W.delta_to_pt(np.array(delta), gg))


def ref(gg):
    gamma0 = gg / G
    return gamma0, math.sqrt(1 - 1 / gamma0 ** 2)


def sample_states(gg, n=6, seed=7, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        d = scale * 1e-3 * rng.standard_normal()
        out.append(np.array([scale * 2e-3 * rng.standard_normal(), scale * 2e-4 * rng.standard_normal(),
                             scale * 2e-3 * rng.standard_normal(), scale * 2e-4 * rng.standard_normal(),
                             1e-2 * rng.standard_normal(), pt_of(d, gg)]))
    return out


def jacobian(fun, z0, eps=1e-30):
    """Exact Jacobian by complex-step differentiation of a map built on the
    complex-valued oracle build."""
    J = np.zeros((6, 6))
    for j in range(6):
        zc = np.array(z0, dtype=np.complex128)
        zc[j] += 1j * eps
        out = fun(zc)
        J[:, j] = out.imag / eps
    return J


OMEGA6 = np.kron(np.eye(3), np.array([[0.0, 1.0], [-1.0, 0.0]]))


# ---------------------------------------------------------------------------
# orbit sub-flows against Hamilton's equations
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_drift_matches_hamilton_ode(gg):
    for z0 in sample_states(gg):
        zo, rc = oracle.subflow("drift", G, gg, z0, 2.3)
        assert rc == 0
        zr = integrate("drift", z0, 2.3, G, gg)
        assert np.abs(zo - zr).max() < 2e-14


@pytest.mark.parametrize("eta", [1.0, 1.003, 0.98])
@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_sbend_matches_hamilton_ode(gg, eta):
    h = 2 * math.pi / 16 / 3.0
    for z0 in sample_states(gg, scale=3.0):
        zo, rc = oracle.subflow("sbend", G, gg, z0, 3.0, h=h, eta=eta)
        assert rc == 0
        zr = integrate("sbend", z0, 3.0, G, gg, h=h, eta=eta)
        assert np.abs(zo - zr).max() < 2e-13


@pytest.mark.parametrize("k1", [0.05, -0.05, 0.0, 0.8])
def test_quad_linear_flow_matches_ode(k1):
    gg = 45.5
    for z0 in sample_states(gg, scale=5.0):
        zo, _ = oracle.subflow("quad_linear", G, gg, z0, 0.7, k1=k1)
        zr = integrate("quad_linear", z0, 0.7, G, gg, k1=k1)
        assert np.abs(zo - zr).max() < 1e-14


def test_quad_nonlinear_flow_matches_ode():
    gg = 45.5
    for z0 in sample_states(gg, scale=10.0):
        zo, rc = oracle.subflow("quad_nonlinear", G, gg, z0, 0.7)
        assert rc == 0
        zr = integrate("quad_nonlinear", z0, 0.7, G, gg)
        assert np.abs(zo - zr).max() < 1e-14


def test_multipole_kick_matches_ode():
    gg = 45.5
    for z0 in sample_states(gg, scale=10.0):
        zo, _ = oracle.subflow("kick", G, gg, z0, 0.3, k1=0.05, k2=0.5)
        zr = integrate("kick", z0, 0.3, G, gg, k1=0.05, k2=0.5)
        assert np.abs(zo - zr).max() < 1e-15


# ---------------------------------------------------------------------------
# closed forms and exact properties of the maps
# ---------------------------------------------------------------------------

def test_drift_composition_is_additive():
    gg = 45.5
    for z0 in sample_states(gg):
        a, _ = oracle.subflow("drift", G, gg, z0, 1.25)
        ab, _ = oracle.subflow("drift", G, gg, a, 0.75)
        c, _ = oracle.subflow("drift", G, gg, z0, 2.0)
        assert np.abs(ab - c).max() < 1e-16
        assert ab[1] == z0[1] and ab[3] == z0[3] and ab[5] == z0[5]


def test_sbend_slicing_is_exact_and_origin_preserved():
    gg = 45.5
    ang = 2 * math.pi / 16
    el1 = W.element("sbend", L=3.0, n_slices=1, angle=ang)
    el8 = W.element("sbend", L=3.0, n_slices=8, angle=ang)
    for z0 in sample_states(gg, scale=3.0):
        a, _ = oracle.orbit_map(el1, G, gg, z0)
        b, _ = oracle.orbit_map(el8, G, gg, z0)
        assert np.abs(a - b).max() < 1e-14      # X carries 1/h times the rounding of its bracket
    o, _ = oracle.orbit_map(el8, G, gg, np.zeros(6))
    assert np.abs(o).max() < 1e-15          # eta = 1 preserves the origin (Sec. 3.1)


def test_sbend_px_sym_locus():
    """Eq. (45): entrance Px on the locus Px_sym(X_i) leaves the magnet with the
    same Px."""
    gg = 382.2
    L, ang = 9.45, math.radians(2.225)
    h = ang / L
    gamma0, beta0 = ref(gg)
    n_checked = 0
    for Xi in (-0.05, -0.01, 0.0, 0.02, 0.05):
        for Py in (-2e-4, 0.0, 2e-4):
            for Pt in (-2e-4, 0.0, 2e-4):
                c, s = math.cos(h * L / 2), math.sin(h * L / 2)
                arg = 1 + 2 * Pt / beta0 + Pt ** 2 - Py ** 2 - (1 + h * Xi) ** 2 * c * c
                if arg <= 0:
                    continue          # no real locus at this (X, Py, Pt)
                n_checked += 1
                root = math.sqrt(arg)
                px_sym = c * (root - (1 + h * Xi) * s)
                z0 = np.array([Xi, px_sym, 0.0, Py, 0.0, Pt])
                zf, rc = oracle.subflow("sbend", G, gg, z0, L, h=h, eta=1.0)
                assert rc == 0
                assert abs(zf[1] - px_sym) < 1e-16
    assert n_checked >= 25


def test_sbend_planar_momentum_invariant():
    gg = 45.5
    gamma0, beta0 = ref(gg)
    h = 2 * math.pi / 16 / 3.0
    for z0 in sample_states(gg, scale=3.0):
        zf, _ = oracle.subflow("sbend", G, gg, z0, 3.0, h=h, eta=1.0)
        assert zf[3] == z0[3] and zf[5] == z0[5]          # Py, Pt constants of motion


def test_quad_linear_reduces_to_textbook_thick_quad():
    """At Pt = 0 (P = 1) the linear flow is the textbook thick-quadrupole
    matrix in (X, X') with X' = Px; defocusing plane with cosh/sinh."""
    gg = 45.5
    k1, s = 0.05, 1.0
    kap = math.sqrt(k1)

    def f(zc):
        out, _ = oracle.subflow("quad_linear", G, gg, zc, s, k1=k1, variant="c128")
        return out

    J = jacobian(f, np.zeros(6))
    Mf = np.array([[math.cos(kap * s), math.sin(kap * s) / kap], [-kap * math.sin(kap * s), math.cos(kap * s)]])
    Md = np.array([[math.cosh(kap * s), math.sinh(kap * s) / kap], [kap * math.sinh(kap * s), math.cosh(kap * s)]])
    assert np.abs(J[0:2, 0:2] - Mf).max() < 1e-15
    assert np.abs(J[2:4, 2:4] - Md).max() < 1e-15


def test_dkd_slice_paraxial_matrix():
    """One drift-kick-drift slice at the origin, Pt = 0: D(l/2) K(k1 l) D(l/2)
    with the textbook drift and thin-lens matrices (fixes the D/2-K-D/2 form)."""
    gg = 45.5
    k1, l = 0.05, 0.25
    el = W.element("mult", L=l, n_slices=1, k1=k1)

    def f(zc):
        out, _ = oracle.orbit_map(el, G, gg, zc, variant="c128")
        return out

    J = jacobian(f, np.zeros(6))
    D = np.array([[1.0, l / 2], [0.0, 1.0]])
    Kx = np.array([[1.0, 0.0], [-k1 * l, 1.0]])
    Ky = np.array([[1.0, 0.0], [k1 * l, 1.0]])
    assert np.abs(J[0:2, 0:2] - D @ Kx @ D).max() < 1e-15
    assert np.abs(J[2:4, 2:4] - D @ Ky @ D).max() < 1e-15


@pytest.mark.parametrize("el", [
    W.element("mult", L=0.4, n_slices=1, k1=0.05, k2=0.5),
    W.element("quad_mk", L=0.5, n_slices=1, k1=0.03),
    W.element("quad_mk", L=0.5, n_slices=1, k1=-0.03),
    W.element("sbend", L=3.0, n_slices=1, angle=2 * math.pi / 16),
    W.element("sbend", L=3.0, n_slices=1, angle=2 * math.pi / 16, eta=1.01),
], ids=["dkd", "mk_f", "mk_d", "bk", "bk_eta"])
def test_slice_jacobian_is_symplectic(el):
    gg = 487.0
    for z0 in sample_states(gg, n=4, scale=5.0):
        def f(zc):
            out, _ = oracle.orbit_map(el, G, gg, zc, variant="c128")
            return out
        J = jacobian(f, z0)
        assert np.abs(J.T @ OMEGA6 @ J - OMEGA6).max() < 1e-12


@pytest.mark.parametrize("el", [
    W.element("mult", L=0.4, n_slices=3, k1=0.05, k2=0.5),
    W.element("quad_mk", L=1.0, n_slices=4, k1=0.03),
    W.element("quad_mk", L=1.0, n_slices=4, k1=-0.03),
    W.element("sbend", L=3.0, n_slices=4, angle=2 * math.pi / 16),
], ids=["dkd", "mk_f", "mk_d", "bk"])
def test_symmetric_splits_are_time_reversible(el):
    gg = 45.5
    back = dict(el, L=-el["L"], angle=-el["angle"])    # same curvature, negative length
    for z0 in sample_states(gg, scale=5.0):
        a, _ = oracle.orbit_map(el, G, gg, z0)
        b, _ = oracle.orbit_map(back, G, gg, a)
        assert np.abs(b - z0).max() < 1e-14


@pytest.mark.parametrize("kind,el_kw,ode_kw", [
    ("mult", dict(type="mult", k1=0.05, k2=0.5), dict(k1=0.05, k2=0.5)),
    ("quad", dict(type="quad_mk", k1=0.05), dict(k1=0.05)),
    ("quad", dict(type="quad_mk", k1=-0.05), dict(k1=-0.05)),
])
def test_split_maps_converge_at_second_order(kind, el_kw, ode_kw):
    gg = 45.5
    L = 1.0
    z0 = np.array([3e-3, 3e-4, -2e-3, 2e-4, 0.0, pt_of(2e-3, gg)])
    zr = integrate(kind, z0, L, G, gg, **ode_kw)
    errs = []
    for N in (2, 4, 8, 16):
        el = W.element(L=L, n_slices=N, **el_kw)
        zo, _ = oracle.orbit_map(el, G, gg, z0)
        errs.append(np.abs(zo - zr)[:4].max())
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    for r in ratios:
        assert 3.6 < r < 4.4, (errs, ratios)


# ---------------------------------------------------------------------------
# precession vector and spin integration
# ---------------------------------------------------------------------------

def test_omega_on_axis_dipole_is_minus_G_gamma_h():
    for gg in (45.5, 487.0):
        ang, L = 2 * math.pi / 16, 3.0
        el = W.element("sbend", L=L, n_slices=4, angle=ang)
        om, rc = oracle.omega(el, G, gg, np.zeros(6))
        assert rc == 0
        assert abs(om[1] + gg * ang / L) < 1e-13 * gg and abs(om[0]) == 0 and abs(om[2]) == 0
        # constant Omega: every level and the Romberg limit are the exact
        # rotation by -G gamma theta about y, for any slicing and order
        for K in (0, 1, 2):
            _, _, levels, Q, _ = oracle.element_detail(el, G, gg, np.zeros(6), [0, 1, 0], K)
            phi = -gg * ang
            assert abs(Q[0] - math.cos(phi / 2)) < 1e-14 and abs(Q[2] - math.sin(phi / 2)) < 1e-14


@pytest.mark.parametrize("el", [
    W.element("mult", L=0.5, n_slices=2, k1=0.05, k2=0.5),
    W.element("quad_mk", L=1.0, n_slices=4, k1=-0.03),
    W.element("sbend", L=3.0, n_slices=4, angle=2 * math.pi / 16, eta=1.002),
], ids=["mult", "quad", "sbend"])
def test_omega_matches_tbmt_decomposition(el):
    """Eq. (6b) against the textbook split of Thomas-BMT into the field parts
    transverse (1 + G gamma) and parallel (1 + G) to the velocity, with the
    field taken as the curl of the element's vector potential."""
    gg = 487.0
    gamma0, beta0 = ref(gg)
    kind = {"mult": "mult", "quad_mk": "quad", "sbend": "sbend"}[el["type"]]
    h = el["angle"] / el["L"] if el["type"] == "sbend" else 0.0
    for z0 in sample_states(gg, scale=30.0):
        om, rc = oracle.omega(el, G, gg, z0)
        ref_om = precession(kind, z0, G, gamma0, beta0, h=h, eta=el["eta"], k1=el["k1"], k2=el["k2"])
        assert np.abs(om - ref_om).max() < 1e-14 * max(1.0, np.abs(ref_om).max())


def test_midplane_bend_closed_form_and_romberg_rates():
    """Mid-plane particle in a sector bend: Omega is along y, so every level is
    a rotation about y by the trapezoid sum, whose exact limit follows from
    Eq. (10b) and Eq. (6b): Phi = -G gamma h L + (1 + G gamma)(psi(L) - psi_i),
    psi = asin(Px/P_alpha).  Trapezoid error ~ N^-2, one Romberg step ~ N^-4,
    two ~ N^-6."""
    gg = 487.0
    gamma0, beta0 = ref(gg)
    L, ang = 3.0, 0.4
    h = ang / L
    z0 = np.array([4e-3, 5e-4, 0.0, 0.0, 0.0, pt_of(1e-3, gg)])
    Pt = z0[5]
    gamma = gamma0 * (1 + beta0 * Pt)
    Pa = math.sqrt(1 + 2 * Pt / beta0 + Pt * Pt)
    zf, _ = oracle.subflow("sbend", G, gg, z0, L, h=h, eta=1.0)
    phi = -G * gamma * h * L + (1 + G * gamma) * (math.asin(zf[1] / Pa) - math.asin(z0[1] / Pa))
    res = {}
    for K in (0, 1, 2):
        errs = []
        for N in (8, 16, 32):
            el = W.element("sbend", L=L, n_slices=N, angle=ang)
            _, _, levels, Q, _ = oracle.element_detail(el, G, gg, z0, [0, 1, 0], K)
            # all levels are rotations about y
            assert np.abs(levels[:, [1, 3]]).max() < 1e-15
            ang_k = 2 * math.atan2(Q[2], Q[0])
            d = (ang_k - phi + math.pi) % (2 * math.pi) - math.pi
            errs.append(abs(d))
        res[K] = errs
    r0 = res[0][0] / res[0][1]
    r1 = res[1][0] / res[1][1]
    r2 = res[2][0] / res[2][1]
    assert 3.7 < r0 < 4.3, res
    assert 13 < r1 < 19, res
    assert 45 < r2 < 80, res


def _element_spin_error(el, gg, z0, S0, K, Sref):
    _, S, _, Q, _ = oracle.element_detail(el, G, gg, z0, S0, K)
    return np.linalg.norm(S - Sref)


def test_spin_converges_to_tbmt_ode_at_paper_rates():
    gold = json.load(open(os.path.join(GOLDEN, "paper_single_element.json")))
    p = gold["test_particle"]
    gamma_total = gold["proton_energy_GeV"]["value"] / 0.93827208816
    gg = G * math.sqrt(1 + gamma_total ** 2)          # 200 GeV/c: gamma = sqrt(1 + (p/m)^2)
    z0 = np.array([p["X"], p["Px"], p["Y"], p["Py"], p["T"], pt_of(p["delta"], gg)])
    S0 = np.array(p["spin"]) / np.linalg.norm(p["spin"])
    brho = gold["proton_energy_GeV"]["value"] / 0.299792458
    # IR quadrupole
    k1 = gold["ir_quad"]["b2_T_per_m"] / brho
    Lq = gold["ir_quad"]["L"]
    _, Sref = integrate("quad", z0, Lq, G, gg, k1=k1, S0=S0)
    e = {(N, K): _element_spin_error(W.element("quad_mk", L=Lq, n_slices=N, k1=k1), gg, z0, S0, K, Sref)
         for N in (4, 8, 16, 256, 512) for K in (0, 1, 2)}
    assert 3.8 < e[(4, 0)] / e[(8, 0)] < 4.2                     # PWC slope -2
    assert 14 < e[(4, 1)] / e[(8, 1)] < 18                       # one Romberg step: slope -4
    assert 50 < e[(4, 2)] / e[(8, 2)] < 80                       # two steps: slope -6
    decades = math.log10(e[(4, 0)] / e[(4, 2)])
    assert 3.5 < decades < 4.5                                   # "four-decade reduction"
    assert e[(512, 0)] < e[(4, 2)] < e[(256, 0)]                 # "some four hundred slices"
    # arc dipole, one Romberg step, slope about -4 between 8 and 64 slices
    Ld, ang = gold["rhic_dipole"]["L"], math.radians(gold["rhic_dipole"]["angle_deg"])
    _, Sref = integrate("sbend", z0, Ld, G, gg, h=ang / Ld, eta=1.0, S0=S0)
    e8 = _element_spin_error(W.element("sbend", L=Ld, n_slices=8, angle=ang), gg, z0, S0, 1, Sref)
    e64 = _element_spin_error(W.element("sbend", L=Ld, n_slices=64, angle=ang), gg, z0, S0, 1, Sref)
    slope = math.log(e64 / e8) / math.log(8)
    assert -5.0 < slope < -3.8
    p8 = _element_spin_error(W.element("sbend", L=Ld, n_slices=8, angle=ang), gg, z0, S0, 0, Sref)
    p64 = _element_spin_error(W.element("sbend", L=Ld, n_slices=64, angle=ang), gg, z0, S0, 0, Sref)
    assert -2.1 < math.log(p64 / p8) / math.log(8) < -1.9


def test_paper_best_reference_agrees_with_ode():
    """The paper's 'best' setting (256 slices, 3 Romberg iterations) is at the
    ODE solution to round-off for the quadrupole."""
    gg = 382.2
    z0, S0 = W.footnote_particle(gg)
    z0, S0 = z0[:, 0], S0[:, 0]
    k1 = 70.0 / (200 / 0.299792458)
    zr, Sr = integrate("quad", z0, 1.83, G, gg, k1=k1, S0=S0)
    err = _element_spin_error(W.element("quad_mk", L=1.83, n_slices=256, k1=k1), gg, z0, S0, 3, Sr)
    assert err < 1e-14


def test_unit_norms_per_element():
    gg = 487.0
    for el in (W.element("quad_mk", L=1.0, n_slices=4, k1=0.03),
               W.element("mult", L=0.2, n_slices=4, k2=0.5),
               W.element("sbend", L=3.0, n_slices=4, angle=0.5)):
        for z0 in sample_states(gg, scale=3.0):
            S0 = np.array([0.3, 0.9, -math.sqrt(1 - 0.81 - 0.09)])
            _, S, _, Q, _ = oracle.element_detail(el, G, gg, z0, S0, 2)
            assert abs(np.linalg.norm(Q) - 1) < 1e-15
            assert abs(np.linalg.norm(S) - 1) < 1e-15


# ---------------------------------------------------------------------------
# ring-level facts
# ---------------------------------------------------------------------------

def test_ring_without_snakes_on_axis_rotates_by_2pi_G_gamma():
    gg = 45.5
    ring = W.with_spin_order(W.toy_ring(gg), 2)
    z = np.zeros((6, 1))
    S = np.array([[1.0], [0.0], [0.0]])
    _, S1, _ = oracle.track(ring, z, S, 1, 2)
    a = -2 * math.pi * gg
    # rotation about y by a: x' = x cos a + s sin a, s' = -x sin a + s cos a
    assert abs(S1[0, 0] - math.cos(a)) < 1e-12
    assert abs(S1[2, 0] + math.sin(a)) < 1e-12
    assert abs(S1[1, 0]) < 1e-15


@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_two_snakes_give_spin_tune_one_half(gg):
    """Two snakes with orthogonal horizontal axes (+-45 deg) half a ring apart
    make the on-axis one-turn rotation a rotation by pi (spin tune 1/2)
    about the vertical, whatever G gamma is (Sec. 5: spin tune exactly 1/2,
    equilibrium polarisation vertical)."""
    ring = W.with_spin_order(W.rhic_like_ring(gg, n_cells=12), 2)
    z = np.zeros((6, 3))
    S = np.eye(3)
    _, S1, _ = oracle.track(ring, z, S, 1, 2)
    R = S1        # columns: images of x, y, s
    assert abs(np.trace(R) - (-1.0)) < 1e-11          # 1 + 2 cos(pi) = -1
    _, S2, _ = oracle.track(ring, z, S1, 1, 2)
    assert np.abs(S2 - np.eye(3)).max() < 1e-11        # two turns: identity
    # the stable spin direction is vertical: R y = y
    assert abs(R[1, 1] - 1.0) < 1e-11


def test_lost_particle_keeps_entrance_state():
    gg = 45.5
    ring = W.with_spin_order(W.toy_ring(gg), 2)
    z = np.zeros((6, 2))
    z[1, 1] = 1.2          # |Px| > P: longitudinal momentum imaginary
    S = np.zeros((3, 2)); S[1] = 1.0
    z1, S1, lost = oracle.track(ring, z, S, 3, 2)
    assert list(lost) == [0, 1]
    assert np.array_equal(z1[:, 1], z[:, 1]) and np.array_equal(S1[:, 1], S[:, 1])


def test_invalid_lattice_rejected():
    ring = W.toy_ring(45.5)          # 4 slices
    assert oracle.check_lattice(ring, 2)
    assert not oracle.check_lattice(ring, 3)
    with pytest.raises(ValueError):
        oracle.track(ring, np.zeros((6, 1)), np.array([[0.0], [1.0], [0.0]]), 1, 3)


def test_oracle_rounding_noise_against_extended_precision():
    """The FP64 oracle agrees with its own long-double build on the toy ring
    after 100 turns far below the parity tolerance; this bounds the oracle's
    rounding noise."""
    w = W.workload("toy_ring_1024")
    z, S = W.gaussian_particles(64, 45.5, seed=1501)
    z64, S64, _ = oracle.track(w["ring"], z, S, 100, 2)
    z80, S80, _ = oracle.track(w["ring"], z, S, 100, 2, variant="f80")
    assert np.abs(z64[:4] - z80[:4].astype(float)).max() < 1e-12
    assert np.abs(S64 - S80.astype(float)).max() < 1e-12


@pytest.mark.parametrize("gg", [45.5, 487.0])
@pytest.mark.parametrize("K", [2, 4])
def test_oracle_rounding_noise_on_the_full_rhic_like_ring(gg, K):
    """The FP64 oracle against its long-double build on the full 108-cell ring
    (Sec. 5's ring with snakes), particles sampled across the 10^5-particle
    bench ensemble.  After one turn the two agree to a few 1e-12.  After 100
    turns they differ by up to 3e-10 m in X and T and 1e-8 in the spin: the
    exact bend map of Eq. (10) forms X as (Ps - eta - A_f)/(eta h), with
    1/(eta h) = 206 m amplifying every rounding of Ps ~ 1, and those errors
    accumulate over the 1728 bend slices of each turn.  This is the rounding
    floor under which no FP64 tracker can be held to the oracle on this ring
    after 100 turns."""
    w = W.workload("rhic_like_1e5", spin_order=K, Ggamma0=gg)
    z, S = W.gaussian_particles(w["n_particles"], gg, seed=w["seed"])
    idx = np.linspace(0, w["n_particles"] - 1, 16).astype(int)
    z, S = z[:, idx], S[:, idx]
    z64, S64, _ = oracle.track(w["ring"], z, S, 1, K)
    z80, S80, _ = oracle.track(w["ring"], z, S, 1, K, variant="f80")
    assert np.abs(z64 - z80.astype(float)).max() < 1e-11
    assert np.abs(S64 - S80.astype(float)).max() < 1e-11
    z64, S64, l64 = oracle.track(w["ring"], z64, S64, 99, K)
    z80, S80, l80 = oracle.track(w["ring"], z80, S80, 99, K, variant="f80")
    assert l64.sum() == 0 and l80.sum() == 0
    dz = np.abs(z64 - z80.astype(float)).max(axis=1)
    assert dz[0] < 1e-9 and dz[2] < 1e-10 and dz[4] < 2e-9, dz        # X, Y, T in m
    assert dz[1] < 2e-11 and dz[3] < 2e-12 and dz[5] == 0.0, dz       # Px, Py; Pt is constant
    assert np.abs(S64 - S80.astype(float)).max() < 3e-8


def _thick_lens(el):
    """Textbook linear 4x4 transverse matrix (X, Px, Y, Py) of an element on
    momentum (P = 1): drifts, thick quadrupoles (cos/cosh), a sector dipole
    with design field (horizontal rotation by its angle, vertical drift)."""
    L = el["L"]
    drift = np.array([[1.0, L], [0.0, 1.0]])
    if el["type"] == "drift":
        return np.block([[drift, np.zeros((2, 2))], [np.zeros((2, 2)), drift]])
    if el["type"] in ("quad_mk", "mult"):
        k = math.sqrt(abs(el["k1"]))
        f = np.array([[math.cos(k * L), math.sin(k * L) / k], [-k * math.sin(k * L), math.cos(k * L)]])
        d = np.array([[math.cosh(k * L), math.sinh(k * L) / k], [k * math.sinh(k * L), math.cosh(k * L)]])
        mx, my = (f, d) if el["k1"] > 0 else (d, f)
        return np.block([[mx, np.zeros((2, 2))], [np.zeros((2, 2)), my]])
    if el["type"] == "sbend":
        th = el["angle"]
        rho = L / th
        mx = np.array([[math.cos(th), rho * math.sin(th)], [-math.sin(th) / rho, math.cos(th)]])
        return np.block([[mx, np.zeros((2, 2))], [np.zeros((2, 2)), drift]])
    raise KeyError(el["type"])


def test_cell_linear_map_and_phase_advance_match_thick_lens_matrices():
    """One FODO cell of the toy ring on momentum: with matrix-kick
    quadrupoles the oracle's transverse Jacobian (complex step) equals the
    product of the textbook thick-lens matrices to 1e-12; with the ring's
    drift-kick-drift quadrupoles (4 slices) the phase advances agree to the
    split's O(ds^2) (0.5%).  The ring tunes (8 cells) come out near 1.72 and
    0.49."""
    gg = 45.5
    ring = W.toy_ring(gg)
    cell = ring["elements"][:8]
    assert [e["type"] for e in cell] == ["mult", "drift", "sbend", "drift"] * 2

    def mu(M2):
        return math.acos(0.5 * np.trace(M2))

    M = np.eye(4)
    for e in cell:
        M = _thick_lens(e) @ M
    for quad_type, tol in (("quad_mk", None), ("mult", 5e-3)):
        els = [dict(e, type=quad_type) if e["type"] == "mult" else e for e in cell]

        def one_cell(zc):
            for e in els:
                zc, rc = oracle.orbit_map(e, G, gg, zc, variant="c128")
                assert rc == 0
            return zc

        J = jacobian(one_cell, np.zeros(6))[:4, :4]
        if tol is None:
            assert np.abs(J - M).max() < 1e-12, np.abs(J - M).max()
        else:
            for i in (0, 2):
                assert abs(mu(J[i:i + 2, i:i + 2]) / mu(M[i:i + 2, i:i + 2]) - 1.0) < tol
    nux, nuy = (8 * mu(M[i:i + 2, i:i + 2]) / (2 * math.pi) for i in (0, 2))
    assert abs(nux - 1.724) < 0.01 and abs(nuy - 0.491) < 0.01, (nux, nuy)
