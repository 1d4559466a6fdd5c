"""Independent reference for the oracle: direct numerical integration of
Hamilton's equations and of the Thomas-BMT equation.

Nothing here reuses the paper's closed-form maps.  Hamilton's equations are
obtained by symbolic differentiation (sympy) of the Hamiltonians of Sec. 2.1
and Sec. 3 (Eq. (3) with the element's vector potential, and the split pieces
of Eqs. (21) and (29)); the field b = B/(B rho) is obtained as the curl of the
vector potential in the curved frame; the precession vector is written in the
textbook decomposition of Thomas-BMT into the parts of the field transverse
and parallel to the velocity, (1 + G gamma) b_perp + (1 + G) b_par, plus the
rotation of the Frenet-Serret frame.  The ODEs are integrated with scipy's
DOP853 at tight tolerances.
"""
from __future__ import annotations

import functools
import math

import numpy as np
import sympy as sp
from scipy.integrate import solve_ivp

X, Px, Y, Py, T, Pt = sp.symbols("X Px Y Py T Pt", real=True)
VARS = (X, Px, Y, Py, T, Pt)
beta0_s, h_s, eta_s, k1_s, k2_s = sp.symbols("beta0 h eta k1 k2", real=True)


def _P2():
    return 1 + 2 * Pt / beta0_s + Pt ** 2


def _Ps():
    return sp.sqrt(_P2() - Px ** 2 - Py ** 2)


def _V(kind):
    """Scaled potential term V = -(q/p0)(1 + hX) A_s of Eq. (3) for each element
    family (Eqs. (7), (28); quadrupole of Sec. 3.3)."""
    if kind == "drift":
        return sp.Integer(0)
    if kind == "sbend":
        return eta_s / 2 * (1 + h_s * X) ** 2
    if kind in ("mult", "quad"):
        w = sp.expand((X + sp.I * Y) ** 2)
        w3 = sp.expand((X + sp.I * Y) ** 3)
        return sp.re(k1_s / 2 * w) + sp.re(k2_s / 2 / 3 * w3)
    raise KeyError(kind)


def hamiltonian(kind):
    """Hamiltonian of an element (or of a split piece)."""
    P = sp.sqrt(_P2())
    if kind == "drift":
        return -_Ps() + Pt / beta0_s
    if kind == "sbend":
        return -(1 + h_s * X) * _Ps() + _V("sbend") + Pt / beta0_s
    if kind in ("mult", "quad"):
        return -_Ps() + Pt / beta0_s + _V("mult")
    if kind == "quad_linear":      # Eq. (21b)
        return (Px ** 2 + Py ** 2) / (2 * P) + k1_s / 2 * (X ** 2 - Y ** 2)
    if kind == "quad_nonlinear":   # Eq. (21c)
        return -_Ps() - (Px ** 2 + Py ** 2) / (2 * P) + Pt / beta0_s
    if kind == "kick":
        return _V("mult")
    raise KeyError(kind)


@functools.lru_cache(maxsize=None)
def _vector_field(kind):
    H = hamiltonian(kind)
    rhs = [sp.diff(H, Px), -sp.diff(H, X), sp.diff(H, Py), -sp.diff(H, Y),
           sp.diff(H, Pt), -sp.diff(H, T)]
    return sp.lambdify((VARS, beta0_s, h_s, eta_s, k1_s, k2_s), rhs, "numpy")


@functools.lru_cache(maxsize=None)
def _field_funcs(kind):
    """b = B/(B rho) from the curl of A_s in the curved frame with scale
    factor hs = 1 + hX: b_x = -(1/hs) dV/dY, b_y = (1/hs) dV/dX, where
    V = -(1 + hX) A_s/(B rho)."""
    V = _V("sbend" if kind == "sbend" else ("drift" if kind == "drift" else "mult"))
    hs = 1 + (h_s * X if kind == "sbend" else 0)
    bx = -sp.diff(V, Y) / hs
    by = sp.diff(V, X) / hs
    return sp.lambdify((VARS, h_s, eta_s, k1_s, k2_s), [bx, by], "numpy")


def precession(kind, z, G, gamma0, beta0, h=0.0, eta=1.0, k1=0.0, k2=0.0):
    """Thomas-BMT precession vector with s as independent variable.
    Field split into components along the velocity (factor 1 + G) and
    transverse to it (factor 1 + G gamma); dt/ds = (1 + hX)/v_s; plus the
    rotation rate of the curved frame about y (+h)."""
    bx, by = _field_funcs(kind)(tuple(z), h, eta, k1, k2)
    b = np.array([bx, by, 0.0], dtype=float)
    P2 = 1 + 2 * z[5] / beta0 + z[5] ** 2
    P = math.sqrt(P2)
    Ps = math.sqrt(P2 - z[1] ** 2 - z[3] ** 2)
    u = np.array([z[1], z[3], Ps]) / P
    gamma = gamma0 * (1 + beta0 * z[5])
    b_par = np.dot(u, b) * u
    b_perp = b - b_par
    hs = 1 + (h * z[0] if kind == "sbend" else 0.0)
    om = -(hs / Ps) * ((1 + G * gamma) * b_perp + (1 + G) * b_par)
    if kind == "sbend":
        om = om + np.array([0.0, h, 0.0])
    return om


def integrate(kind, z0, s, G, Ggamma0, h=0.0, eta=1.0, k1=0.0, k2=0.0, S0=None,
              rtol=1e-13, atol=1e-16):
    """Integrate the orbit (and the spin if S0 is given) over a length s."""
    gamma0 = Ggamma0 / G
    beta0 = math.sqrt(1 - 1 / gamma0 ** 2)
    f = _vector_field(kind)
    z0 = np.asarray(z0, dtype=float).reshape(6)
    spin_kind = {"quad_linear": None, "quad_nonlinear": None, "kick": None}.get(kind, kind)
    if kind == "quad":
        spin_kind = "quad"

    def rhs(_s, y):
        z = y[:6]
        dz = np.array(f(tuple(z), beta0, h, eta, k1, k2), dtype=float)
        if S0 is None:
            return dz
        om = precession(spin_kind, z, G, gamma0, beta0, h, eta, k1, k2)
        return np.concatenate([dz, np.cross(om, y[6:])])

    y0 = z0 if S0 is None else np.concatenate([z0, np.asarray(S0, float).reshape(3)])
    sol = solve_ivp(rhs, (0.0, s), y0, method="DOP853", rtol=rtol, atol=atol)
    assert sol.success, sol.message
    yf = sol.y[:, -1]
    return (yf[:6], yf[6:]) if S0 is not None else yf
