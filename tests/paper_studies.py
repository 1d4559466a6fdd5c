"""Input grids of the paper's single-element error studies (Sec. 5.2.1), shared
by the oracle tests and the GPU tests: the RHIC arc dipole over horizontal
phase space (Figs. sbendErrsQ, sbendErrsR, sbendErrsQR4M, sbendErrsQR8M) and
the RHIC IR quadrupole over the (X, Y) plane with spins spread over a cap
about the vertical (Fig. quadErrs48QR).  Magnet data come from
tests/golden/paper_single_element.json.  Nothing here tracks a particle."""
from __future__ import annotations

import json
import math
import os

import numpy as np

import workloads as W

M_P = 0.93827208816            # proton mass [GeV]
C_LIGHT = 0.299792458          # [m/ns]; B rho [T m] = p [GeV/c] / C_LIGHT

_GOLDEN = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                      "paper_single_element.json")))
P_GEV = _GOLDEN["proton_energy_GeV"]["value"]          # read as momentum [GeV/c]
GGAMMA = W.G_PROTON * math.hypot(P_GEV / M_P, 1.0)
DIPOLE_L = _GOLDEN["rhic_dipole"]["L"]
DIPOLE_ANGLE = math.radians(_GOLDEN["rhic_dipole"]["angle_deg"])
QUAD_L = _GOLDEN["ir_quad"]["L"]
QUAD_K1 = _GOLDEN["ir_quad"]["b2_T_per_m"] * C_LIGHT / P_GEV


def beta0():
    gamma0 = GGAMMA / W.G_PROTON
    return math.sqrt(1.0 - 1.0 / gamma0 ** 2)


def footnote_spin():
    s = np.array([0.1952, 0.9759, 0.0976])
    return s / np.linalg.norm(s)


def dipole(n_slices):
    return W.single_element_ring(W.element("sbend", L=DIPOLE_L, n_slices=n_slices, angle=DIPOLE_ANGLE), GGAMMA)


def ir_quad(n_slices):
    return W.single_element_ring(W.element("quad_mk", L=QUAD_L, n_slices=n_slices, k1=QUAD_K1), GGAMMA)


def dipole_grid(Py, Pt, nx=21, npx=61):
    """Figs. sbendErrsQR4M/QR8M: X in +-5 cm, Px in +-6 mrad at fixed Py, Pt,
    the footnote spin.  Returns (z [6, nx*npx], S, X [nx], PX [npx])."""
    X = np.linspace(-0.05, 0.05, nx)
    PX = np.linspace(-6e-3, 6e-3, npx)
    XX, PP = np.meshgrid(X, PX, indexing="ij")
    n = XX.size
    z = np.zeros((6, n))
    z[0], z[1], z[3], z[5] = XX.ravel(), PP.ravel(), Py, Pt
    S = np.tile(footnote_spin()[:, None], (1, n))
    return z, S, X, PX


def px_sym(X, Py, Pt):
    """Eq. (dpx0): the entrance Px that the dipole returns unchanged at its exit
    (NaN where there is none)."""
    h = DIPOLE_ANGLE / DIPOLE_L
    c, s = math.cos(0.5 * h * DIPOLE_L), math.sin(0.5 * h * DIPOLE_L)
    P2 = 1.0 + 2.0 * Pt / beta0() + Pt * Pt
    arg = P2 - Py * Py - (1.0 + h * X) ** 2 * c * c
    with np.errstate(invalid="ignore"):
        return c * (np.sqrt(arg) - (1.0 + h * X) * s)


def cap_spins(alpha_deg, m):
    """m quasi-random unit vectors (a Fibonacci lattice) on the cap of half-angle
    alpha about the vertical y axis; one vertical spin for alpha = 0."""
    if alpha_deg == 0:
        return np.array([[0.0], [1.0], [0.0]])
    a = math.radians(alpha_deg)
    k = np.arange(m) + 0.5
    cy = 1.0 - (1.0 - math.cos(a)) * k / m
    ph = k * math.pi * (3.0 - math.sqrt(5.0))
    r = np.sqrt(1.0 - cy * cy)
    return np.stack([r * np.cos(ph), cy, r * np.sin(ph)])


def quad_grid(alpha_deg, m=8, n=21):
    """Fig. quadErrs48QR: X, Y in +-20 mm with Px = Py = Pt = 0, every point
    with each spin of the cap.  Returns (z, S, n_points, n_spins); particle
    j * n_points + k is grid point k with spin j."""
    g = np.linspace(-20e-3, 20e-3, n)
    XX, YY = np.meshgrid(g, g, indexing="ij")
    spins = cap_spins(alpha_deg, m)
    npt, ms = XX.size, spins.shape[1]
    z = np.zeros((6, npt * ms))
    S = np.zeros((3, npt * ms))
    for j in range(ms):
        z[0, j * npt:(j + 1) * npt] = XX.ravel()
        z[2, j * npt:(j + 1) * npt] = YY.ravel()
        S[:, j * npt:(j + 1) * npt] = spins[:, j:j + 1]
    return z, S, npt, ms


def spin_error_map(S, Sref, npt, ms):
    """|S - S_ref| per particle, averaged over the spins of each grid point."""
    return np.linalg.norm(S - Sref, axis=0).reshape(ms, npt).mean(axis=0)
