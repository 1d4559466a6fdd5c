"""Pins of the oracle's midpoint spin schemes: piece-wise constant rotations
with Omega at the middle of each slice (Sec. 4.1, Eq. (37)), either between
two half-slices ("half-DKD, spin rotation, half-DKD") or between the two
halves of a drift-kick or matrix-kick slice's central kick ("half-drift,
half-kick, spin rotation, half-kick, half-drift"), Sec. 5.3 and
Fig. oneTurnSpinErrs.  Pinned against the midpoint rule's textbook error on
the mid-plane bend's closed form, Thomas-BMT integrated along Hamilton's
equations, and the paper's one-turn and multi-turn comparisons of drift-kick
and bend-kick / matrix-kick integration."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from ode_reference import integrate

G = W.G_PROTON
S0 = np.array([0.3, 0.2, math.sqrt(1 - 0.13)])
SCHEMES = [oracle.MID_HALF, oracle.MID_KICK]


def test_midpoint_rule_on_the_midplane_bend():
    """Mid-plane particle in a sector bend: all rotations are about y, so the
    element angle is the midpoint-rule sum of Omega_y, whose exact value is
    Phi = -G gamma h L + (1 + G gamma)(psi(L) - psi_i) (Eqs. (10b), (6b)).
    The midpoint error falls as N^-2 and is -1/2 of the trapezoid rule's
    (Romberg order 0 on the slice edges) for a smooth integrand."""
    gg = 487.0
    gamma0 = gg / G
    beta0 = math.sqrt(1 - 1 / gamma0 ** 2)
    L, ang = 3.0, 0.4
    h = ang / L
    z0 = np.array([4e-3, 5e-4, 0.0, 0.0, 0.0, float(W.delta_to_pt(np.array(1e-3), gg))])
    gamma = gamma0 * (1 + beta0 * z0[5])
    Pa = math.sqrt(1 + 2 * z0[5] / beta0 + z0[5] ** 2)
    zf, _ = oracle.subflow("sbend", G, gg, z0, L, h=h, eta=1.0)
    phi = -G * gamma * h * L + (1 + G * gamma) * (math.asin(zf[1] / Pa) - math.asin(z0[1] / Pa))

    def err(N, K):
        _, _, _, Q, rc = oracle.element_detail(W.element("sbend", L=L, n_slices=N, angle=ang), G, gg, z0,
                                               [0, 1, 0], K)
        assert rc == 0
        assert abs(Q[1]) < 1e-15 and abs(Q[3]) < 1e-15
        return (2 * math.atan2(Q[2], Q[0]) - phi + math.pi) % (2 * math.pi) - math.pi

    for K in SCHEMES:
        e = [err(N, K) for N in (8, 16, 32)]
        assert all(3.9 < e[i] / e[i + 1] < 4.1 for i in range(2)), e
        for N in (16, 32):
            assert -0.52 < err(N, K) / err(N, 0) < -0.48


@pytest.mark.parametrize("el", [
    W.element("mult", L=1.0, n_slices=4, k1=0.3, k2=3.0),
    W.element("quad_mk", L=1.0, n_slices=4, k1=-0.4),
    W.element("teapot", L=3.0, n_slices=4, angle=0.2, eta=1.01),
], ids=["dkd", "mk", "teapot"])
def test_kick_placement_keeps_the_slice_map_and_half_slices_double_it(el):
    """Splitting the central kick leaves the orbit map of each slice (the two
    half-kicks commute); the half-slice placement gives the orbit of twice as
    many slices."""
    gg = 45.5
    z0 = np.array([3e-3, 3e-4, -2e-3, 2e-4, 1e-3, float(W.delta_to_pt(np.array(2e-3), gg))])
    zk, _, _, _, rc = oracle.element_detail(el, G, gg, z0, S0, oracle.MID_KICK)
    assert rc == 0
    z1, _ = oracle.orbit_map(el, G, gg, z0)
    assert np.abs(zk - z1).max() < 1e-16 + 1e-13 * (el["type"] == "teapot")
    zh, _, _, _, _ = oracle.element_detail(el, G, gg, z0, S0, oracle.MID_HALF)
    z2, _ = oracle.orbit_map(dict(el, n_slices=2 * el["n_slices"]), G, gg, z0)
    assert np.abs(zh - z2).max() < 1e-16 + 1e-13 * (el["type"] == "teapot")


@pytest.mark.parametrize("kind,el_kw,ode_kw", [
    ("mult", dict(type="mult", k1=0.5, k2=5.0), dict(k1=0.5, k2=5.0)),
    ("quad", dict(type="quad_mk", k1=0.5), dict(k1=0.5)),
    ("sbend", dict(type="sbend", angle=0.2, eta=1.01), dict(h=0.2, eta=1.01)),
], ids=["dkd", "mk", "sbend"])
@pytest.mark.parametrize("K", SCHEMES)
def test_midpoint_spin_converges_at_second_order(kind, el_kw, ode_kw, K):
    """Against Thomas-BMT integrated along Hamilton's equations, the midpoint
    schemes converge as N^-2."""
    gg = 45.5
    z0 = np.array([3e-3, 3e-4, -2e-3, 2e-4, 0.0, float(W.delta_to_pt(np.array(2e-3), gg))])
    _, Sref = integrate(kind, z0, 1.0, G, gg, S0=S0, **ode_kw)
    errs = []
    for N in (8, 16, 32):
        _, S, _, _, rc = oracle.element_detail(W.element(L=1.0, n_slices=N, **el_kw), G, gg, z0, S0, K)
        assert rc == 0
        errs.append(np.linalg.norm(S - Sref))
    assert all(3.7 < errs[i] / errs[i + 1] < 4.3 for i in range(2)), errs


def mean_spin_error(S, Sref):
    """Delta S of Sec. 5.3: the mean over the ensemble of |S_j - S_j(ref)|."""
    return float(np.linalg.norm(S - Sref, axis=0).mean())


@pytest.mark.parametrize("gg,min_ratio", [(45.5, 100.0), (487.0, 10.0)])
def test_one_turn_errors_drift_kick_against_bend_kick(gg, min_ratio):
    """Sec. 5.3, Fig. oneTurnSpinErrs: one turn of the RHIC-scale ring without
    Romberg steps, against bend-kick / matrix-kick integration with n_b = 256
    and three Romberg iterations.  Drift-kick integration (TEAPOT bends,
    drift-kick-drift quadrupoles) with either spin placement converges as
    n_b^-2; bend-kick / matrix-kick integration with the same n_b is more
    than two decades more accurate than the drift-kick placement at G gamma0
    = 45.5 (the paper reports two and a half for RHIC) and more than one at
    487; the half-slice placement, whose drift-kick orbit is that of 2 n_b
    slices, is four times closer."""
    base = W.rhic_like_ring(gg)
    z, S = W.gaussian_particles(16, gg, seed=3)
    _, Sref, lost = oracle.track(W.with_slices(base, 256), z, S, 1, 3)
    assert not lost.any()
    dk = W.drift_kick_ring(base)
    res = {}
    for nb in (4, 8, 16):
        _, s_kick, _ = oracle.track(W.with_slices(dk, nb), z, S, 1, oracle.MID_KICK)
        _, s_half, _ = oracle.track(W.with_slices(dk, nb), z, S, 1, oracle.MID_HALF)
        _, s_bkmk, _ = oracle.track(W.with_slices(base, nb), z, S, 1, oracle.MID_HALF)
        res[nb] = [mean_spin_error(s, Sref) for s in (s_kick, s_half, s_bkmk)]
    for nb in (4, 8):
        for j in range(3):
            assert 3.6 < res[nb][j] / res[2 * nb][j] < 4.4, res
    for nb, (e_kick, e_half, e_bkmk) in res.items():
        assert e_half < e_kick                       # half-slices: the orbit of 2 n_b slices
        assert e_kick > min_ratio * e_bkmk, res
        assert e_half > 0.25 * min_ratio * e_bkmk, res


def test_spin_errors_over_turns_order_of_the_integrators():
    """Sec. 5.3, Fig. spinErrVsTurns, on the RHIC-scale ring at G gamma0 = 45.5
    with n_b = 4: the TEAPOT split (drift-kick placement) lies above
    bend-kick / matrix-kick with the trapezoid rule, which lies above
    bend-kick / matrix-kick with Romberg iterations, at every turn: the
    TEAPOT error more than two decades above, the Romberg error at least two
    times below (its gain shrinks as the split error of the orbit, which
    Romberg does not remove, accumulates)."""
    gg = 45.5
    base = W.rhic_like_ring(gg)
    z, S = W.gaussian_particles(16, gg, seed=5)
    ref_ring = W.with_slices(base, 128)
    runs = {"teapot": (W.with_slices(W.drift_kick_ring(base), 4), oracle.MID_KICK),
            "bkmk_pwc": (W.with_slices(base, 4), 0),
            "bkmk_romberg": (W.with_slices(base, 4), 2)}
    state = {k: (z, S) for k in runs}
    zr, Sr = z, S
    for turn in range(8):
        zr, Sr, _ = oracle.track(ref_ring, zr, Sr, 1, 3)
        errs = {}
        for k, (ring, K) in runs.items():
            zk, Sk, lk = oracle.track(ring, *state[k], 1, K)
            assert not lk.any()
            state[k] = (zk, Sk)
            errs[k] = mean_spin_error(Sk, Sr)
        assert errs["teapot"] > 100 * errs["bkmk_pwc"], (turn, errs)
        assert errs["bkmk_pwc"] > 2 * errs["bkmk_romberg"], (turn, errs)


def test_midpoint_validation():
    # any slice count, but not the fourth-order maps
    assert oracle.check_lattice(W.single_element_ring(W.element("mult", L=1.0, n_slices=3, k1=0.1), 45.5),
                                oracle.MID_KICK)
    assert not oracle.check_lattice(W.single_element_ring(W.element("mult", L=1.0, n_slices=3, k1=0.1), 45.5), 1)
    for K in SCHEMES:
        ring = W.single_element_ring(W.element("quad_mk", L=1.0, n_slices=4, k1=0.1, split_order=4), 45.5)
        assert not oracle.check_lattice(ring, K)
    assert not oracle.check_lattice(W.toy_ring(45.5), -3)


@pytest.mark.parametrize("el", [
    W.element("solenoid", L=2.0, n_slices=1, k1=0.3),
    W.element("rbend", L=3.0, n_slices=1, angle=0.1, e1=0.02, fringe=1),
    W.element("thin_mult", n_slices=1, k1=0.2, k2=5.0),
], ids=["solenoid", "rbend", "thin_lens"])
@pytest.mark.parametrize("K", SCHEMES)
def test_midpoint_converges_to_the_romberg_limit_on_every_element_kind(el, K):
    """Both midpoint placements converge as N^-2 to the limit that three
    Romberg iterations on 256 slices reach (the same integral of Eq. (37))
    on the solenoid (with its fringe kicks), the rectangular bend (with its
    rotations and fringe kicks) and the thin lens."""
    gg = 45.5
    z0 = np.array([2e-3, 3e-4, -2e-3, 2e-4, 0.0, float(W.delta_to_pt(np.array(1e-3), gg))])
    _, Sref, _, _, rc = oracle.element_detail(dict(el, n_slices=256), G, gg, z0, S0, 3)
    assert rc == 0
    errs = []
    for N in (8, 16, 32):
        _, S, _, _, rc = oracle.element_detail(dict(el, n_slices=N), G, gg, z0, S0, K)
        assert rc == 0
        errs.append(np.linalg.norm(S - Sref))
    assert all(3.6 < errs[i] / errs[i + 1] < 4.4 for i in range(2)), errs
