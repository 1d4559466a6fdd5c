"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only *describes* inputs: ring lattices as lists of element dicts
and particle ensembles as float64 arrays.  It holds none of the tracking
arithmetic (no orbit map, no precession vector, no quaternion); both the CPU
oracle and the CUDA library receive exactly the same element list and the same
uploaded doubles.

Element dict keys (all lengths in m, strengths in the paper's normalised form
b/(B rho), Sec. 2.1 and Sec. 3):

    type       "drift" | "mult" (drift-kick-drift multipole, Sec. 3.4)
               | "quad_mk" (matrix-kick quadrupole, Sec. 3.3)
               | "sbend" (exact bend-kick sector bend, Sec. 3.1)
               | "snake" (thin spin rotator, Sec. 5)
               | "teapot" (sector bend integrated by the TEAPOT drift-kick
                 split, Sec. 3.6: curved drift, kick, curved drift)
               | "thin_mult" (thin lens, Sec. 3.5: L = 0, k1 and k2 hold the
                 integrated strengths k1 L [m^-1] and k2 L [m^-2]; n_slices
                 samples the spin along the kick)
    L          length
    n_slices   number of integration slices (spin-carrying elements)
    k1         quadrupole gradient b2/(B rho)            [m^-2]
    k2         sextupole strength  B''/(B rho) (MAD k2)  [m^-3]
    angle      bend angle h*L of a sector bend           [rad]
    eta        field ratio eta = b1/(h B rho), Eq. (9)
    snake_phi  snake axis angle from the longitudinal axis, in the x-s plane
    snake_mu   snake rotation angle
    fringe     1: thin fringe spin kicks at both ends of a mult, quad_mk,
               sbend or teapot (Sec. 4.5, Eq. (skfringe)); 0: hard edges
               without kicks
    split_order  orbit slice map of a mult, quad_mk or teapot: 2 = the symmetric split
               of Eq. (27), 4 = its fourth-order Yoshida composition (Sec. 3.3)
    e1         rbend: the beam meets the entrance face at angle/2 + e1 and the
               exit face at -angle/2 + e1 (0: symmetric rectangular bend)
    (rbend: "rbend", Sec. 3.2: L is the magnet length along its Cartesian
    axis, angle the total bend, eta the field factor; its thin-fringe orbit
    map is always applied, its Eq. (skfringeRB) spin kicks when fringe = 1)
    (solenoid: "solenoid" with k1 = b0/(B rho), MAD's ks, Sec. 3.7; its
    thin-pancake fringe kicks, Sec. 4.4, are always part of the element)

The ring description dict: {"G", "Ggamma0", "elements": [...], "name"}.

Particle ensembles follow the Gaussian recipe of the toy proton ring: sigma_x =
sigma_y = 1 mm, sigma_px = sigma_py = 0.1 mrad, sigma_T = 1 cm, sigma_delta =
1e-3 (relative momentum deviation), spins along y.  The energy coordinate Pt of
Eq. (2) is obtained from delta through the definition of Pt and of the scale
momentum p0 (input preparation, not part of the tracked map).
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np

G_PROTON = 1.7928

ELEMENT_TYPES = ("drift", "mult", "quad_mk", "sbend", "snake", "solenoid", "rbend", "teapot", "thin_mult")
SPIN_TYPES = ("mult", "quad_mk", "sbend", "solenoid", "rbend", "teapot", "thin_mult")


def element(type: str, L: float = 0.0, n_slices: int = 1, k1: float = 0.0,
            k2: float = 0.0, angle: float = 0.0, eta: float = 1.0,
            snake_phi: float = 0.0, snake_mu: float = 0.0, name: str = "",
            fringe: int = 0, split_order: int = 2, e1: float = 0.0) -> Dict:
    if type not in ELEMENT_TYPES:
        raise ValueError(f"unknown element type {type!r}")
    return dict(type=type, L=float(L), n_slices=int(n_slices), k1=float(k1),
                k2=float(k2), angle=float(angle), eta=float(eta),
                snake_phi=float(snake_phi), snake_mu=float(snake_mu),
                name=name or type, fringe=int(fringe), split_order=int(split_order), e1=float(e1))


def slices_for_order(base: int, spin_order: int) -> int:
    """Smallest multiple of 2**spin_order that is >= base (Romberg needs the
    slice count divisible by 2**k, Sec. 4.3); any count >= 1 for the midpoint
    schemes (negative spin_order)."""
    m = 1 << max(spin_order, 0)
    return max(m, ((base + m - 1) // m) * m)


RING_FORMAT = "spintrack-ring-1"
_ELEMENT_KEYS = ("type", "L", "n_slices", "k1", "k2", "angle", "eta", "snake_phi", "snake_mu", "name", "fringe",
                 "split_order", "e1")


def save_ring(ring: Dict, path: str) -> None:
    """Write a ring as JSON: {"format", "name", "G", "Ggamma0", "elements": [...]}
    with every element field written out (the lattice description file)."""
    import json
    out = {"format": RING_FORMAT, "name": ring.get("name", ""), "G": float(ring["G"]),
           "Ggamma0": float(ring["Ggamma0"]),
           "elements": [{k: element(**{kk: e[kk] for kk in _ELEMENT_KEYS if kk in e})[k] for k in _ELEMENT_KEYS}
                        for e in ring["elements"]]}
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


def load_ring(path: str) -> Dict:
    """Read a ring written by save_ring (or by hand).  Unknown element types or
    fields raise ValueError; omitted fields take element()'s defaults."""
    import json
    with open(path) as f:
        d = json.load(f)
    if d.get("format") != RING_FORMAT:
        raise ValueError(f"{path}: not a {RING_FORMAT} file")
    els = []
    for i, e in enumerate(d["elements"]):
        extra = set(e) - set(_ELEMENT_KEYS)
        if extra:
            raise ValueError(f"{path}: element {i}: unknown fields {sorted(extra)}")
        els.append(element(**e))
    return dict(name=d.get("name", ""), G=float(d["G"]), Ggamma0=float(d["Ggamma0"]), elements=els)


def with_spin_order(ring: Dict, spin_order: int) -> Dict:
    """Copy of `ring` whose spin-carrying elements have slice counts valid for
    Romberg order `spin_order`."""
    out = dict(ring)
    out["elements"] = []
    for e in ring["elements"]:
        e = dict(e)
        if e["type"] in SPIN_TYPES:
            e["n_slices"] = slices_for_order(e["n_slices"], spin_order)
        out["elements"].append(e)
    return out


def with_fringes(ring: Dict, on: int = 1) -> Dict:
    """Copy of `ring` with the thin fringe spin kicks of Sec. 4.5 switched on
    (or off) at both ends of every multipole, quadrupole and sector bend."""
    out = dict(ring)
    out["elements"] = [dict(e, fringe=int(on)) if e["type"] in ("mult", "quad_mk", "sbend", "teapot") else dict(e)
                       for e in ring["elements"]]
    out["name"] = ring["name"] + ("_fringes" if on else "")
    return out


def with_split_order(ring: Dict, order: int) -> Dict:
    """Copy of `ring` whose multipoles and matrix-kick quadrupoles use the
    second-order (2) or fourth-order (4) slice map (Sec. 3.3)."""
    out = dict(ring)
    out["elements"] = [dict(e, split_order=int(order)) if e["type"] in ("mult", "quad_mk") else dict(e)
                       for e in ring["elements"]]
    out["name"] = ring["name"] + (f"_split{order}" if order != 2 else "")
    return out


def drift_kick_ring(ring: Dict) -> Dict:
    """Copy of `ring` integrated by drift-kick splits only (the integrators the
    paper compares against, Sec. 3.4, 3.6, 5.3): matrix-kick quadrupoles
    become drift-kick-drift multipoles of the same gradient and exact sector
    bends become TEAPOT bends of the same angle and field."""
    conv = {"quad_mk": "mult", "sbend": "teapot"}
    out = dict(ring)
    out["elements"] = [dict(e, type=conv.get(e["type"], e["type"])) for e in ring["elements"]]
    out["name"] = ring["name"] + "_drift_kick"
    return out


def with_thin_sextupoles(ring: Dict) -> Dict:
    """Copy of `ring` whose thick sextupoles (mult elements without a
    quadrupole part) are thin lenses of the same integrated strength
    (Sec. 3.5) between two drifts of half their length."""
    out = dict(ring)
    els = []
    for e in ring["elements"]:
        if e["type"] == "mult" and e["k1"] == 0.0 and e["L"] > 0.0:
            half = element("drift", L=0.5 * e["L"], name=e["name"] + "_d")
            els += [half, element("thin_mult", n_slices=e["n_slices"], k2=e["k2"] * e["L"], name=e["name"]),
                    dict(half)]
        else:
            els.append(dict(e))
    out["elements"] = els
    out["name"] = ring["name"] + "_thin_sext"
    return out


def with_slices(ring: Dict, n_slices: int) -> Dict:
    """Copy of `ring` with every spin-carrying element cut into n_slices
    slices (the paper's n_b)."""
    out = dict(ring)
    out["elements"] = [dict(e, n_slices=int(n_slices)) if e["type"] in SPIN_TYPES else dict(e)
                       for e in ring["elements"]]
    return out


def reference(Ggamma0: float, G: float = G_PROTON):
    """(gamma0, beta0) of the scale momentum for a given naive spin tune."""
    gamma0 = Ggamma0 / G
    beta0 = math.sqrt(1.0 - 1.0 / (gamma0 * gamma0))
    return gamma0, beta0


# ---------------------------------------------------------------------------
# rings
# ---------------------------------------------------------------------------

def toy_ring(Ggamma0: float = 45.5, n_cells: int = 8, k1: float = 0.05,
             quad_slices: int = 4, bend_slices: int = 4) -> Dict:
    """Toy proton ring: 8 FODO cells of QF(1 m, k1=+0.05, DKD) D(2) B(3 m,
    2pi/16, BK) D(2) QD(1 m, k1=-0.05, DKD) D(2) B D(2); 64 elements, 128 m."""
    ang = 2.0 * math.pi / (2 * n_cells)
    els = []
    for c in range(n_cells):
        els += [
            element("mult", L=1.0, n_slices=quad_slices, k1=+k1, name=f"QF{c}"),
            element("drift", L=2.0, name=f"D{c}a"),
            element("sbend", L=3.0, n_slices=bend_slices, angle=ang, name=f"B{c}a"),
            element("drift", L=2.0, name=f"D{c}b"),
            element("mult", L=1.0, n_slices=quad_slices, k1=-k1, name=f"QD{c}"),
            element("drift", L=2.0, name=f"D{c}c"),
            element("sbend", L=3.0, n_slices=bend_slices, angle=ang, name=f"B{c}b"),
            element("drift", L=2.0, name=f"D{c}d"),
        ]
    return dict(name="toy_proton_ring", G=G_PROTON, Ggamma0=float(Ggamma0), elements=els)


def solenoid_ring(Ggamma0: float = 45.5, ks: float = 0.05, n_cells: int = 8,
                  sol_slices: int = 8) -> Dict:
    """The toy ring of toy_ring() with the first 2 m drift of cells 0 and
    n_cells/2 replaced by 2 m solenoids of strength ks = b0/(B rho) [1/m]
    (opposite signs, so that the transverse coupling of the two partly
    cancels, as for a detector solenoid and its compensator)."""
    ring = toy_ring(Ggamma0, n_cells=n_cells)
    els = ring["elements"]
    for c, sign in ((0, +1.0), (n_cells // 2, -1.0)):
        i = 8 * c + 1
        assert els[i]["type"] == "drift" and els[i]["L"] == 2.0
        els[i] = element("solenoid", L=2.0, n_slices=sol_slices, k1=sign * ks, name=f"SOL{c}")
    ring["name"] = "toy_ring_solenoids"
    return ring


def rbend_ring(Ggamma0: float = 45.5, n_cells: int = 8, e1: float = 0.0, fringe: int = 0,
               bend_slices: int = 4) -> Dict:
    """The toy ring of toy_ring() with every 3 m sector bend replaced by a
    rectangular bend of the same angle and the same reference arc (magnet
    length = chord 2 rho sin(angle/2), rho = 3 m / angle), Sec. 3.2."""
    ring = toy_ring(Ggamma0, n_cells=n_cells)
    els = []
    for e in ring["elements"]:
        if e["type"] == "sbend":
            ang = e["angle"]
            rho = e["L"] / ang
            e = element("rbend", L=2.0 * rho * math.sin(0.5 * ang), n_slices=bend_slices, angle=ang, e1=e1,
                        fringe=fringe, name=e["name"].replace("B", "RB"))
        els.append(e)
    ring["elements"] = els
    ring["name"] = "toy_ring_rbends"
    return ring


def rhic_like_ring(Ggamma0: float = 45.5, n_cells: int = 108, k1: float = 0.03,
                   k2: float = 0.5, base_slices: int = 4, sext_slices: int = 2,
                   snakes: bool = True, quad_type: str = "quad_mk") -> Dict:
    """RHIC-scale synthetic ring: n_cells FODO cells of
    QF(1, +k1, MK) SF(0.2, +k2, DKD) D(1.8) B(3) D(2) B(3) D(2)
    QD(1, -k1, MK) SD(0.2, -k2, DKD) D(1.8) B(3) D(2) B(3) D(2),
    26 m per cell, 4*n_cells sector dipoles of angle 2pi/(4 n_cells), and two
    ideal Siberian snakes (pi rotations about horizontal axes at +-45 deg from
    the longitudinal axis): one at s=0, one after cell n_cells/2 - 1."""
    ang = 2.0 * math.pi / (4 * n_cells)
    els = []
    half = n_cells // 2
    if snakes:
        els.append(element("snake", snake_phi=+math.pi / 4, snake_mu=math.pi, name="SNK1"))
    for c in range(n_cells):
        els += [
            element(quad_type, L=1.0, n_slices=base_slices, k1=+k1, name=f"QF{c}"),
            element("mult", L=0.2, n_slices=sext_slices, k2=+k2, name=f"SF{c}"),
            element("drift", L=1.8, name=f"D{c}a"),
            element("sbend", L=3.0, n_slices=base_slices, angle=ang, name=f"B{c}a"),
            element("drift", L=2.0, name=f"D{c}b"),
            element("sbend", L=3.0, n_slices=base_slices, angle=ang, name=f"B{c}b"),
            element("drift", L=2.0, name=f"D{c}c"),
            element(quad_type, L=1.0, n_slices=base_slices, k1=-k1, name=f"QD{c}"),
            element("mult", L=0.2, n_slices=sext_slices, k2=-k2, name=f"SD{c}"),
            element("drift", L=1.8, name=f"D{c}d"),
            element("sbend", L=3.0, n_slices=base_slices, angle=ang, name=f"B{c}c"),
            element("drift", L=2.0, name=f"D{c}e"),
            element("sbend", L=3.0, n_slices=base_slices, angle=ang, name=f"B{c}d"),
            element("drift", L=2.0, name=f"D{c}f"),
        ]
        if snakes and c == half - 1:
            els.append(element("snake", snake_phi=-math.pi / 4, snake_mu=math.pi, name="SNK2"))
    return dict(name=f"rhic_like_{n_cells}cells", G=G_PROTON, Ggamma0=float(Ggamma0), elements=els)


def batched_jobs(n_jobs: int = 64, seed: int = 20240603, turns: int = 500,
                 min_cells: int = 8, max_cells: int = 108,
                 min_particles: int = 1000, max_particles: int = 100000) -> List[Dict]:
    """Uneven batch: rings with U{min_cells..max_cells} cells (the RHIC-like
    layout scaled to the cell count, snakes only for an even cell count),
    G*gamma0 ~ U[45.5, 487], particle counts log-uniform in
    [min_particles, max_particles], every job `turns` turns."""
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n_jobs):
        cells = int(rng.integers(min_cells, max_cells + 1))
        gg = float(rng.uniform(45.5, 487.0))
        n = int(round(10.0 ** rng.uniform(math.log10(min_particles), math.log10(max_particles))))
        ring = rhic_like_ring(Ggamma0=gg, n_cells=cells, snakes=(cells % 2 == 0))
        jobs.append(dict(ring=ring, n_particles=n, turns=turns, seed=seed * 1000 + j))
    return jobs


def single_element_ring(el: Dict, Ggamma0: float, G: float = G_PROTON) -> Dict:
    return dict(name="single_" + el["type"], G=G, Ggamma0=float(Ggamma0), elements=[dict(el)])


def count_passes(ring: Dict, n_particles: int, n_turns: int) -> int:
    """Particle-element passes: one particle through one element (drifts and
    snakes included)."""
    return len(ring["elements"]) * n_particles * n_turns


# ---------------------------------------------------------------------------
# particles
# ---------------------------------------------------------------------------

def delta_to_pt(delta: np.ndarray, Ggamma0: float, G: float = G_PROTON) -> np.ndarray:
    """Energy coordinate Pt of Eq. (2) for relative momentum deviation delta:
    with P = p/p0 = 1 + delta and m c^2/(p0 c) = 1/(beta0 gamma0),
    Pt = sqrt(P^2 + 1/(beta0 gamma0)^2) - 1/beta0."""
    gamma0, beta0 = reference(Ggamma0, G)
    inv_bg = 1.0 / (beta0 * gamma0)
    return np.sqrt((1.0 + delta) ** 2 + inv_bg * inv_bg) - 1.0 / beta0


DEFAULT_SIGMAS = dict(x=1e-3, px=1e-4, y=1e-3, py=1e-4, t=1e-2, delta=1e-3)


def gaussian_particles(n: int, Ggamma0: float, seed: int, sigmas: Dict = None,
                       G: float = G_PROTON, spin=(0.0, 1.0, 0.0), cut: float = None):
    """6D Gaussian ensemble.  Returns (z, S): z is float64 [6, n] in the order
    (X, Px, Y, Py, T, Pt) of Eq. (1); S is float64 [3, n] (x, y, s components).
    `cut` truncates each normal deviate at +-cut sigma (resampling)."""
    s = dict(DEFAULT_SIGMAS)
    if sigmas:
        s.update(sigmas)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((6, n))
    if cut is not None:
        bad = np.abs(g) > cut
        while bad.any():
            g[bad] = rng.standard_normal(int(bad.sum()))
            bad = np.abs(g) > cut
    z = np.empty((6, n), dtype=np.float64)
    z[0] = s["x"] * g[0]
    z[1] = s["px"] * g[1]
    z[2] = s["y"] * g[2]
    z[3] = s["py"] * g[3]
    z[4] = s["t"] * g[4]
    z[5] = delta_to_pt(s["delta"] * g[5], Ggamma0, G)
    S = np.zeros((3, n), dtype=np.float64)
    S[0], S[1], S[2] = spin
    return z, S


def cap_spins(n: int, alpha: float, seed: int) -> np.ndarray:
    """Unit spins uniformly distributed on the cap of opening angle alpha about
    the vertical y axis (quasi-random cap sampling used for the quadrupole
    spin-error maps of Sec. 5.2).  Uses the area-uniform parametrisation
    cos(theta) ~ U[cos(alpha), 1]."""
    rng = np.random.default_rng(seed)
    ct = rng.uniform(math.cos(alpha), 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    S = np.empty((3, n))
    S[0] = st * np.cos(ph)
    S[1] = ct
    S[2] = st * np.sin(ph)
    return S


# The paper's single-particle test case (Sec. 5.2, footnote on the
# single-element error study): X = 1 mm, Px = 0.1 mrad, Py = -0.2 mrad,
# delta = 1e-3, Y = T = 0, spin ~ (0.1952, 0.9759, 0.0976).
def footnote_particle(Ggamma0: float, G: float = G_PROTON):
    z = np.array([[1e-3], [1e-4], [0.0], [-2e-4], [0.0],
                  [float(delta_to_pt(np.array(1e-3), Ggamma0, G))]])
    s = np.array([0.1952, 0.9759, 0.0976])
    s = s / np.linalg.norm(s)
    return z, s.reshape(3, 1)


# Named workloads (the five benchmark configurations, by what they are).
def workload(name: str, spin_order: int = 2, Ggamma0: float = None):
    """Returns dict(ring, n_particles, turns, spin_order, seed)."""
    if name == "toy_ring_1024":
        ring = toy_ring(45.5 if Ggamma0 is None else Ggamma0)
        return dict(ring=with_spin_order(ring, spin_order), n_particles=1024,
                    turns=100, spin_order=spin_order, seed=1501)
    if name == "rhic_like_1e5":
        ring = rhic_like_ring(45.5 if Ggamma0 is None else Ggamma0)
        return dict(ring=with_spin_order(ring, spin_order), n_particles=100000,
                    turns=1000, spin_order=spin_order, seed=3450)
    if name == "rhic_like_spin_map":
        # learned one-turn spin map: training pairs along the orbits of 4e4
        # Gaussian particles (cut at 3 sigma) over 100 turns (4e6 pairs);
        # use on 1e4 particles x 1e4 turns of stroboscopic averaging; errors
        # measured on 1024 particles at turn 1000
        ring = rhic_like_ring(45.5 if Ggamma0 is None else Ggamma0)
        return dict(ring=with_spin_order(ring, spin_order), n_particles=10000,
                    turns=10000, spin_order=spin_order, seed=3452, cut=3.0,
                    train_particles=40000, train_turns=100, train_seed=777,
                    steps=30000, batch=32768, lr=2e-3, degree=3, eval_particles=1024, eval_turns=1000)
    if name == "rhic_like_1e6_mixed":
        ring = rhic_like_ring(45.5 if Ggamma0 is None else Ggamma0)
        return dict(ring=with_spin_order(ring, spin_order), n_particles=1000000,
                    turns=1000, spin_order=spin_order, seed=3451)
    raise KeyError(name)

