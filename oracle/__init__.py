"""CPU oracle for spin-orbit tracking -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference leg
of `bench.py` may import this package.  The CUDA library never loads it and the
product path has no CPU fallback.

`oracle.c` is a plain FP64 C transcription of the paper's method (see its
header for the section/equation map).  The same source is compiled three ways:

    f64   double          -- the oracle proper
    f80   long double     -- extended precision, used only to measure the
                             oracle's own rounding noise
    c128  double complex  -- complex-step derivatives (exact Jacobians)

`opcount.cpp` compiles the same source once more with a scalar that tallies
every floating-point operation on particle data (the method's algorithmic
work per pass, used for the roofline's numerator).

`mlp.py` holds the FP64 NumPy reference of the learned one-turn spin map.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "oracle.c")

_VARIANTS = {
    "f64": ("double", np.float64),
    "f80": ("long double", np.longdouble),
    "c128": ("double complex", np.complex128),
}

TYPE_CODES = {"drift": 0, "mult": 1, "quad_mk": 2, "sbend": 3, "snake": 4, "solenoid": 5, "rbend": 6,
              "teapot": 7, "thin_mult": 8}

# spin_order values of the midpoint (piece-wise constant) schemes; 0..6 are
# Romberg orders over slice-edge samples
MID_HALF = -1   # each slice as two half-slices, the spin rotation between them
MID_KICK = -2   # second-order drift-kick / matrix-kick slices: between the halves of the central kick

_lock = threading.Lock()
_libs = {}


class OrcElement(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("n_slices", ctypes.c_int32),
                ("L", ctypes.c_double), ("k1", ctypes.c_double), ("k2", ctypes.c_double),
                ("angle", ctypes.c_double), ("eta", ctypes.c_double),
                ("snake_phi", ctypes.c_double), ("snake_mu", ctypes.c_double),
                ("fringe", ctypes.c_int32), ("split_order", ctypes.c_int32), ("e1", ctypes.c_double)]


_OPC_LIB = os.path.join(_BUILD, "liboracle_opcount.so")
OP_NAMES = ("add", "mul", "div", "sqrt", "sincos", "tan", "asin", "sinh_cosh")


def _lib_path(variant: str) -> str:
    return os.path.join(_BUILD, f"liboracle_{variant}.so")


def build(force: bool = False) -> None:
    """Compile the three oracle variants with gcc (-O2, no FMA contraction, no
    fast-math, OpenMP over particles)."""
    os.makedirs(_BUILD, exist_ok=True)
    for variant, (ctype, _) in _VARIANTS.items():
        out = _lib_path(variant)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", f"-DORACLE_REAL={ctype}", _SRC, "-o", out + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)
    out = _OPC_LIB
    cpp = os.path.join(_HERE, "opcount.cpp")
    if force or not os.path.exists(out) or os.path.getmtime(out) < max(os.path.getmtime(_SRC), os.path.getmtime(cpp)):
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-I", _HERE, cpp, "-o", out + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)


def _lib(variant: str = "f64"):
    with _lock:
        if variant not in _libs:
            build()
            lib = ctypes.CDLL(_lib_path(variant))
            vp = ctypes.c_void_p
            lib.orc_real_size.restype = ctypes.c_int
            lib.orc_track.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_long, vp, vp, vp, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int]
            lib.orc_track.restype = ctypes.c_int
            lib.orc_element_detail.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp, vp,
                                               ctypes.c_int, vp, vp]
            lib.orc_element_detail.restype = ctypes.c_int
            lib.orc_orbit_map.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp]
            lib.orc_orbit_map.restype = ctypes.c_int
            lib.orc_subflow.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, vp,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double]
            lib.orc_subflow.restype = ctypes.c_int
            lib.orc_omega.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp, vp]
            lib.orc_solenoid_fringe.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                vp, vp]
            lib.orc_solenoid_fringe.restype = ctypes.c_int
            lib.orc_element_fringe.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, vp, vp]
            lib.orc_element_fringe.restype = ctypes.c_int
            lib.orc_omega.restype = ctypes.c_int
            lib.orc_check_lattice.argtypes = [vp, ctypes.c_int, ctypes.c_int]
            lib.orc_check_lattice.restype = ctypes.c_int
            dt = _VARIANTS[variant][1]
            assert lib.orc_real_size() == np.dtype(dt).itemsize, variant
            _libs[variant] = lib
        return _libs[variant]


def elements_array(elements):
    arr = (OrcElement * max(1, len(elements)))()
    for i, e in enumerate(elements):
        arr[i] = OrcElement(TYPE_CODES[e["type"]], int(e["n_slices"]), e["L"], e["k1"], e["k2"],
                            e["angle"], e["eta"], e["snake_phi"], e["snake_mu"], int(e.get("fringe", 0)), int(e.get("split_order", 2)),
                            float(e.get("e1", 0.0)))
    return arr


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def track(ring, z, S, n_turns, spin_order, lost=None, variant="f64", n_threads=0):
    """Track particles (z [6,n], S [3,n]) through `ring` for n_turns turns with
    Romberg order spin_order (or one of the midpoint schemes MID_HALF,
    MID_KICK).  Returns new arrays (z, S, lost)."""
    dt = _VARIANTS[variant][1]
    z = np.ascontiguousarray(np.array(z, dtype=dt))
    S = np.ascontiguousarray(np.array(S, dtype=dt))
    n = z.shape[1]
    lost = np.zeros(n, np.uint8) if lost is None else np.ascontiguousarray(np.array(lost, np.uint8))
    els = elements_array(ring["elements"])
    rc = _lib(variant).orc_track(els, len(ring["elements"]), ring["G"], ring["Ggamma0"], n,
                                 _ptr(z), _ptr(S), _ptr(lost), int(n_turns), int(spin_order),
                                 int(n_threads))
    if rc != 0:
        raise ValueError("oracle: invalid lattice for this spin order")
    return z, S, lost


def element_detail(el, G, Ggamma0, z6, S3, spin_order, variant="f64"):
    """One particle through one element: returns (z6, S3, levels[K+1,4], Q[4], rc)."""
    dt = _VARIANTS[variant][1]
    z6 = np.ascontiguousarray(np.array(z6, dtype=dt).reshape(6))
    S3 = np.ascontiguousarray(np.array(S3, dtype=dt).reshape(3))
    levels = np.zeros((max(spin_order, 0) + 1, 4), dtype=dt)
    Q = np.zeros(4, dtype=dt)
    rc = _lib(variant).orc_element_detail(elements_array([el]), G, Ggamma0, _ptr(z6), _ptr(S3),
                                          int(spin_order), _ptr(levels), _ptr(Q))
    if rc < 0:
        raise ValueError("oracle: invalid element for this spin order")
    return z6, S3, levels, Q, rc


def orbit_map(el, G, Ggamma0, z6, variant="f64"):
    dt = _VARIANTS[variant][1]
    z6 = np.ascontiguousarray(np.array(z6, dtype=dt).reshape(6))
    rc = _lib(variant).orc_orbit_map(elements_array([el]), G, Ggamma0, _ptr(z6))
    return z6, rc


SUBFLOWS = {"drift": 0, "kick": 1, "quad_linear": 2, "quad_nonlinear": 3, "sbend": 4, "solenoid": 5,
            "rbend_body": 6, "rbend_rotation": 7, "rbend_fringe": 8, "curved_drift": 9, "teapot_kick": 10}


def subflow(which, G, Ggamma0, z6, s, k1=0.0, k2=0.0, h=0.0, eta=1.0, variant="f64"):
    dt = _VARIANTS[variant][1]
    z6 = np.ascontiguousarray(np.array(z6, dtype=dt).reshape(6))
    rc = _lib(variant).orc_subflow(SUBFLOWS[which], G, Ggamma0, _ptr(z6), s, k1, k2, h, eta)
    return z6, rc


def omega(el, G, Ggamma0, z6, variant="f64"):
    dt = _VARIANTS[variant][1]
    z6 = np.ascontiguousarray(np.array(z6, dtype=dt).reshape(6))
    out = np.zeros(3, dtype=dt)
    rc = _lib(variant).orc_omega(elements_array([el]), G, Ggamma0, _ptr(z6), _ptr(out))
    return out, rc


def solenoid_fringe(ks, sign, G, Ggamma0, z6, variant="f64"):
    """Rotation vector of a thin-pancake solenoid fringe (Eq. (solFringe))."""
    dt = _VARIANTS[variant][1]
    z6 = np.ascontiguousarray(np.array(z6, dtype=dt).reshape(6))
    out = np.zeros(3, dtype=dt)
    rc = _lib(variant).orc_solenoid_fringe(float(ks), int(sign), G, Ggamma0, _ptr(z6), _ptr(out))
    return out, rc


def element_fringe(el, sign, G, Ggamma0, z6, variant="f64"):
    """Rotation vector of element el's thin fringe spin kick at its entrance
    (sign +1) or exit (-1): Eq. (skfringe) for dipoles and multipoles,
    Eq. (solFringe) for solenoids.  Returns (w[3], rc)."""
    dt = _VARIANTS[variant][1]
    z6 = np.ascontiguousarray(np.array(z6, dtype=dt).reshape(6))
    out = np.zeros(3, dtype=dt)
    rc = _lib(variant).orc_element_fringe(elements_array([el]), int(sign), G, Ggamma0, _ptr(z6), _ptr(out))
    return out, rc


_opc = None


def op_counts(ring, z, S, n_turns, spin_order):
    """Track (single thread) with the operation-counting build and return
    (counts, z, S, lost): counts maps OP_NAMES to the number of operations on
    particle data (additions include subtractions; sincos counts each sin and
    each cos)."""
    global _opc
    with _lock:
        if _opc is None:
            build()
            lib = ctypes.CDLL(_OPC_LIB)
            vp = ctypes.c_void_p
            lib.opc_track.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_long,
                                      vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
            lib.opc_track.restype = ctypes.c_int
            _opc = lib
    z = np.ascontiguousarray(np.array(z, dtype=np.float64))
    S = np.ascontiguousarray(np.array(S, dtype=np.float64))
    n = z.shape[1]
    lost = np.zeros(n, np.uint8)
    out = np.zeros(len(OP_NAMES), np.uint64)
    rc = _opc.opc_track(elements_array(ring["elements"]), len(ring["elements"]), ring["G"], ring["Ggamma0"], n,
                        _ptr(z), _ptr(S), _ptr(lost), int(n_turns), int(spin_order), _ptr(out))
    if rc != 0:
        raise ValueError("oracle: invalid lattice for this spin order")
    return {k: int(v) for k, v in zip(OP_NAMES, out)}, z, S, lost


def check_lattice(ring, spin_order) -> bool:
    return _lib("f64").orc_check_lattice(elements_array(ring["elements"]),
                                         len(ring["elements"]), int(spin_order)) == 0
