"""Python binding of the spintrack C ABI (include/spintrack.h).

Argument marshalling only: every step of the tracking runs in the CUDA
library `libspintrack.so` built in-tree for sm_103a.  If the library is
missing the import of the binding functions fails loudly; there is no CPU
fallback.  PyTorch is used by callers only for device memory and streams
(pass `tensor.data_ptr()` with `*_is_device=1` and
`torch.cuda.current_stream().cuda_stream`).
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional

import numpy as np

from . import _build

# SPINTRACK_LIB selects another build of the library (e.g. the checked build,
# _build.LIB_CHECKED); it is then loaded as it is, without rebuilding
LIB_PATH = os.environ.get("SPINTRACK_LIB", _build.LIB)

ST_OK, ST_EINVAL, ST_ENOMEM, ST_ECUDA, ST_ETIMEOUT, ST_ESTATE = 0, -1, -2, -3, -4, -5
ST_DRIFT, ST_MULT, ST_QUAD_MK, ST_SBEND, ST_SNAKE, ST_SOLENOID, ST_RBEND, ST_TEAPOT, ST_THIN_MULT = range(9)
ST_FP64, ST_MIXED = 0, 1
# spin_order values of the midpoint schemes (0..4 are Romberg orders)
ST_SPIN_MID_HALF, ST_SPIN_MID_KICK = -1, -2

TYPE_CODES = {"drift": ST_DRIFT, "mult": ST_MULT, "quad_mk": ST_QUAD_MK, "sbend": ST_SBEND, "snake": ST_SNAKE,
              "solenoid": ST_SOLENOID, "rbend": ST_RBEND, "teapot": ST_TEAPOT, "thin_mult": ST_THIN_MULT}
PRECISIONS = {"fp64": ST_FP64, "mixed": ST_MIXED}


class StElement(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("n_slices", ctypes.c_int32), ("L", ctypes.c_double),
                ("k1", ctypes.c_double), ("k2", ctypes.c_double), ("angle", ctypes.c_double),
                ("eta", ctypes.c_double), ("snake_phi", ctypes.c_double), ("snake_mu", ctypes.c_double),
                ("fringe", ctypes.c_int32), ("split_order", ctypes.c_int32), ("e1", ctypes.c_double)]


class StReference(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("Ggamma0", ctypes.c_double)]


class SpinTrackError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"spintrack error {code}: {msg}")
        self.code = code


# Every symbol declared in include/spintrack.h, with its ctypes signature.
_VP = ctypes.c_void_p
SIGNATURES = {
    "st_lattice_create": ([ctypes.POINTER(StElement), ctypes.c_int32, ctypes.POINTER(StReference),
                           ctypes.POINTER(_VP)], ctypes.c_int),
    "st_lattice_destroy": ([_VP], ctypes.c_int),
    "st_ctx_create": ([_VP, ctypes.c_int64, ctypes.c_int32, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "st_ctx_destroy": ([_VP], ctypes.c_int),
    "st_particles_upload": ([_VP, _VP, _VP, ctypes.c_int32], ctypes.c_int),
    "st_lost_upload": ([_VP, _VP, ctypes.c_int32], ctypes.c_int),
    "st_selftest_bounded_wait": ([ctypes.c_double, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "st_track": ([_VP, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "st_spins_download": ([_VP, _VP, _VP, _VP, ctypes.c_int32], ctypes.c_int),
    "st_track_orbit": ([_VP, ctypes.c_int32], ctypes.c_int),
    "st_track_one_turn_map": ([_VP, ctypes.c_int32, _VP, _VP], ctypes.c_int),
    "st_track_average": ([_VP, ctypes.c_int32, ctypes.c_int32, _VP], ctypes.c_int),
    "st_ctx_set_launch": ([_VP, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "st_measure_peaks": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "st_measure_fp32x2_peak": ([ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "st_track_fp64_noalloc": ([ctypes.POINTER(StElement), ctypes.c_int32, ctypes.POINTER(StReference), _VP, _VP,
                               ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _VP], ctypes.c_int),
    "st_tune_slicing": ([ctypes.POINTER(StElement), ctypes.c_int32, ctypes.POINTER(StReference), _VP, _VP,
                         ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_int32),
                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32), _VP], ctypes.c_int),
    "st_batch_create": ([ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, ctypes.c_int32, _VP,
                         ctypes.POINTER(_VP)], ctypes.c_int),
    "st_batch_destroy": ([_VP], ctypes.c_int),
    "st_batch_upload": ([_VP, ctypes.c_int32, _VP, _VP, ctypes.c_int32], ctypes.c_int),
    "st_batch_track": ([_VP, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "st_batch_download": ([_VP, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_int32], ctypes.c_int),
    "st_batch_set_launch": ([_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "st_batch_autotune": ([_VP, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "st_gemm_bf16": ([_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP], ctypes.c_int),
    "st_mlp_param_count": ([], ctypes.c_int64),
    "st_mlp_create": ([ctypes.c_int32, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "st_mlp_destroy": ([_VP], ctypes.c_int),
    "st_mlp_set_params": ([_VP, _VP], ctypes.c_int),
    "st_mlp_get_params": ([_VP, _VP], ctypes.c_int),
    "st_mlp_set_head": ([_VP, _VP, _VP, ctypes.c_double, _VP], ctypes.c_int),
    "st_mlp_set_scale": ([_VP, _VP], ctypes.c_int),
    "st_mlp_fit_head": ([_VP, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_int64, _VP, _VP], ctypes.c_int),
    "st_mlp_make_targets": ([_VP, _VP, _VP, ctypes.c_int64, _VP, _VP], ctypes.c_int),
    "st_mlp_forward": ([_VP, _VP, ctypes.c_int32, _VP], ctypes.c_int),
    "st_mlp_loss_grad": ([_VP, _VP, _VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_float), _VP], ctypes.c_int),
    "st_mlp_loss_grad_residual": ([_VP, _VP, _VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_float), _VP],
                                  ctypes.c_int),
    "st_mlp_adam_step": ([_VP, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float], ctypes.c_int),
    "st_mlp_set_fused_inference": ([_VP, ctypes.c_int32], ctypes.c_int),
    "st_mlp_train": ([_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                      ctypes.POINTER(ctypes.c_float), ctypes.c_float, ctypes.c_float, ctypes.c_float,
                      ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "st_track_surrogate": ([_VP, _VP, ctypes.c_int32, _VP], ctypes.c_int),
    "st_last_error": ([], ctypes.c_char_p),
    "st_version": ([], ctypes.c_char_p),
}

_lib = None


def load(build_if_missing: bool = True):
    """Load libspintrack.so (building it with nvcc if it is missing or stale
    and `build_if_missing`).  Raises if the library cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and LIB_PATH == _build.LIB and not _build.up_to_date():
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"spintrack CUDA library not found at {LIB_PATH}; run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc: int):
    if rc != ST_OK:
        raise SpinTrackError(rc, load().st_last_error().decode())
    return rc


def last_error() -> str:
    return load().st_last_error().decode()


def elements_array(elements: List[Dict]):
    arr = (StElement * len(elements))()
    for i, e in enumerate(elements):
        arr[i] = StElement(TYPE_CODES[e["type"]], int(e["n_slices"]), e["L"], e["k1"], e["k2"], e["angle"],
                           e["eta"], e["snake_phi"], e["snake_mu"], int(e.get("fringe", 0)),
                           int(e.get("split_order", 2)), float(e.get("e1", 0.0)))
    return arr


# ---- thin wrappers with the C names --------------------------------------

def st_lattice_create(elements: List[Dict], G: float, Ggamma0: float) -> int:
    lib = load()
    arr = elements_array(elements)
    ref = StReference(G, Ggamma0)
    out = _VP()
    _check(lib.st_lattice_create(arr, len(elements), ctypes.byref(ref), ctypes.byref(out)))
    return out.value


def st_lattice_destroy(lat: int) -> None:
    _check(load().st_lattice_destroy(lat))


def st_ctx_create(lat: int, n_particles: int, precision: int = ST_FP64, stream: Optional[int] = None) -> int:
    out = _VP()
    _check(load().st_ctx_create(lat, int(n_particles), int(precision), stream, ctypes.byref(out)))
    return out.value


def st_ctx_destroy(ctx: int) -> None:
    _check(load().st_ctx_destroy(ctx))


def st_particles_upload(ctx: int, z_ptr: int, s_ptr: int, src_is_device: int) -> None:
    _check(load().st_particles_upload(ctx, z_ptr, s_ptr, int(src_is_device)))


def st_lost_upload(ctx: int, lost_ptr: int, src_is_device: int) -> None:
    _check(load().st_lost_upload(ctx, lost_ptr, src_is_device))


def st_selftest_bounded_wait(limit_s: float):
    """Run the bounded-wait self-test; returns (rc, elapsed seconds)."""
    el = ctypes.c_double(0.0)
    rc = load().st_selftest_bounded_wait(float(limit_s), ctypes.byref(el))
    return rc, el.value


def st_track(ctx: int, n_turns: int, spin_order: int) -> None:
    _check(load().st_track(ctx, int(n_turns), int(spin_order)))


def st_track_orbit(ctx: int, n_turns: int) -> None:
    _check(load().st_track_orbit(ctx, int(n_turns)))


def st_track_one_turn_map(ctx: int, spin_order: int, q_ref, q_out_ptr: int) -> None:
    qr = np.ascontiguousarray(q_ref, dtype=np.float64)
    _check(load().st_track_one_turn_map(ctx, int(spin_order), qr.ctypes.data, q_out_ptr))


def st_track_average(ctx: int, n_turns: int, spin_order: int, spin_sum_ptr: int) -> None:
    _check(load().st_track_average(ctx, int(n_turns), int(spin_order), spin_sum_ptr))


def st_spins_download(ctx: int, s_ptr: int, z_ptr: Optional[int], lost_ptr: Optional[int],
                      dst_is_device: int) -> None:
    _check(load().st_spins_download(ctx, s_ptr, z_ptr, lost_ptr, int(dst_is_device)))


def st_ctx_set_launch(ctx: int, block_threads: int = 0, turns_per_launch: int = 0) -> None:
    _check(load().st_ctx_set_launch(ctx, int(block_threads), int(turns_per_launch)))


def st_measure_peaks():
    """(fp64_flops, fp32_flops) of the current device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().st_measure_peaks(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def st_measure_fp32x2_peak() -> float:
    """FP32 flop/s of the current device with packed FP32x2 fused multiply-adds."""
    a = ctypes.c_double()
    _check(load().st_measure_fp32x2_peak(ctypes.byref(a)))
    return a.value


def st_track_fp64_noalloc(elements: List[Dict], G: float, Ggamma0: float, state_ptr: int, lost_ptr: int,
                          n_particles: int, n_turns: int, spin_order: int, stream: Optional[int] = None) -> None:
    """Allocation-free FP64 tracking on caller-owned device buffers (see the
    header for the state layout)."""
    arr = elements_array(elements)
    ref = StReference(G, Ggamma0)
    _check(load().st_track_fp64_noalloc(arr, len(elements), ctypes.byref(ref), state_ptr, lost_ptr,
                                        int(n_particles), int(n_turns), int(spin_order), stream))


ST_TUNE_MAX_SLICES, ST_TUNE_MAX_ORDER, ST_TUNE_REF_SLICES, ST_TUNE_REF_ORDER, ST_TUNE_MAX_CANDIDATES = 64, 3, 128, 3, 22


def st_tune_slicing(ring: Dict, z: np.ndarray, S: np.ndarray, spin_error_bound: float) -> Dict:
    """Fastest (n_b, Romberg order) whose one-turn spin error on the sample
    (z [6, n], S [3, n]) stays within the bound (see the header).  Returns
    dict(n_slices, spin_order, dS, ms, table) with table rows (n_b, K, dS, ms)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    arr = elements_array(ring["elements"])
    ref = StReference(ring["G"], ring["Ggamma0"])
    nb, K, nc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    dS, ms = ctypes.c_double(), ctypes.c_float()
    table = np.zeros((ST_TUNE_MAX_CANDIDATES, 4), np.float64)
    _check(load().st_tune_slicing(arr, len(ring["elements"]), ctypes.byref(ref), z.ctypes.data, S.ctypes.data,
                                  z.shape[1], float(spin_error_bound), ctypes.byref(nb), ctypes.byref(K),
                                  ctypes.byref(dS), ctypes.byref(ms), ctypes.byref(nc), table.ctypes.data))
    return dict(n_slices=nb.value, spin_order=K.value, dS=dS.value, ms=ms.value, table=table[:nc.value])


def st_batch_create(lattice_handles: List[int], n_particles: List[int], precision: int = ST_FP64,
                    stream: Optional[int] = None) -> int:
    n = len(lattice_handles)
    lats = (_VP * n)(*lattice_handles)
    ns = (ctypes.c_int64 * n)(*[int(x) for x in n_particles])
    out = _VP()
    _check(load().st_batch_create(lats, ns, n, int(precision), stream, ctypes.byref(out)))
    return out.value


def st_batch_destroy(b: int) -> None:
    _check(load().st_batch_destroy(b))


def st_batch_upload(b: int, job: int, z_ptr: int, s_ptr: int, src_is_device: int) -> None:
    _check(load().st_batch_upload(b, int(job), z_ptr, s_ptr, int(src_is_device)))


def st_batch_track(b: int, n_turns: int, spin_order: int) -> None:
    _check(load().st_batch_track(b, int(n_turns), int(spin_order)))


def st_batch_download(b: int, job: int, s_ptr: int, z_ptr: Optional[int], lost_ptr: Optional[int],
                      dst_is_device: int) -> None:
    _check(load().st_batch_download(b, int(job), s_ptr, z_ptr, lost_ptr, int(dst_is_device)))


def st_batch_set_launch(b: int, block_threads: int = 0, turns_per_launch: int = 0, use_graph: int = -1,
                        variant: int = -1) -> None:
    _check(load().st_batch_set_launch(b, int(block_threads), int(turns_per_launch), int(use_graph), int(variant)))


def st_batch_autotune(b: int, spin_order: int, trial_turns: int = 2):
    blk, tpl, var, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(load().st_batch_autotune(b, int(spin_order), int(trial_turns), ctypes.byref(blk), ctypes.byref(tpl),
                                    ctypes.byref(var), ctypes.byref(ms)))
    return dict(block_threads=blk.value, turns_per_launch=tpl.value, variant=var.value, ms=ms.value)


class Batch:
    """Many independent tracking jobs tracked by one persistent launch."""

    def __init__(self, rings: List[Dict], n_particles: List[int], precision: str = "fp64",
                 stream: Optional[int] = None):
        self.lattices = [Lattice(r) for r in rings]
        self.n = [int(x) for x in n_particles]
        self.handle = st_batch_create([l.handle for l in self.lattices], self.n, PRECISIONS[precision], stream)

    def upload(self, job: int, z: np.ndarray, S: np.ndarray):
        z = np.ascontiguousarray(z, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.float64)
        assert z.shape == (6, self.n[job]) and S.shape == (3, self.n[job])
        st_batch_upload(self.handle, job, z.ctypes.data, S.ctypes.data, 0)

    def track(self, n_turns: int, spin_order: int):
        st_batch_track(self.handle, n_turns, spin_order)

    def download(self, job: int):
        n = self.n[job]
        z = np.empty((6, n))
        S = np.empty((3, n))
        lost = np.empty(n, np.uint8)
        st_batch_download(self.handle, job, S.ctypes.data, z.ctypes.data, lost.ctypes.data, 0)
        return z, S, lost

    def set_launch(self, block_threads=0, turns_per_launch=0, use_graph=-1, variant=-1):
        st_batch_set_launch(self.handle, block_threads, turns_per_launch, use_graph, variant)

    def autotune(self, spin_order: int, trial_turns: int = 2):
        return st_batch_autotune(self.handle, spin_order, trial_turns)

    def close(self):
        if self.handle:
            st_batch_destroy(self.handle)
            self.handle = None
        for l in self.lattices:
            l.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def st_gemm_bf16(A_ptr: int, B_ptr: int, D_ptr: int, M: int, N: int, K: int, bias_ptr: Optional[int],
                 status_ptr: int, stream: Optional[int] = None) -> None:
    _check(load().st_gemm_bf16(A_ptr, B_ptr, D_ptr, int(M), int(N), int(K), bias_ptr, status_ptr, stream))


class MLP:
    """The learned one-turn spin map (device-resident parameters)."""

    def __init__(self, max_batch: int, stream: Optional[int] = None):
        out = _VP()
        _check(load().st_mlp_create(int(max_batch), stream, ctypes.byref(out)))
        self.handle = out.value
        self.n_params = int(load().st_mlp_param_count())

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.shape == (self.n_params,)
        _check(load().st_mlp_set_params(self.handle, p.ctypes.data))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.n_params, np.float32)
        _check(load().st_mlp_get_params(self.handle, p.ctypes.data))
        return p

    def set_head(self, q0, lin, out_scale: float, in_scale):
        q0 = np.ascontiguousarray(q0, dtype=np.float64)
        ins = np.ascontiguousarray(in_scale, dtype=np.float64)
        lp = None
        if lin is not None:
            lin = np.ascontiguousarray(lin, dtype=np.float64).reshape(4, 6)
            lp = lin.ctypes.data
        self._head_keep = (q0, ins, lin)
        _check(load().st_mlp_set_head(self.handle, q0.ctypes.data, lp, float(out_scale), ins.ctypes.data))

    def set_fused_inference(self, on: bool):
        _check(load().st_mlp_set_fused_inference(self.handle, 1 if on else 0))

    def forward(self, x_ptr: int, B: int, q_ptr: int):
        _check(load().st_mlp_forward(self.handle, x_ptr, int(B), q_ptr))

    def set_scale(self, out_scale):
        """Output scales: a number (all components) or four numbers."""
        sc = np.ascontiguousarray(np.broadcast_to(np.asarray(out_scale, dtype=np.float64), (4,)))
        _check(load().st_mlp_set_scale(self.handle, sc.ctypes.data))

    def fit_head(self, degree: int, z_ptr: int, q_ptr: int, n: int, lost_ptr: Optional[int] = None):
        """Returns (coef [4, n_terms], rms [4])."""
        nt = poly_term_count(degree)
        coef = np.empty((4, nt), np.float64)
        rms = np.empty(4, np.float64)
        _check(load().st_mlp_fit_head(self.handle, int(degree), z_ptr, q_ptr, lost_ptr, int(n), coef.ctypes.data,
                                      rms.ctypes.data))
        return coef, rms

    def make_targets(self, z_ptr: int, q_ptr: int, n: int, x_rows_ptr: int, r_rows_ptr: int):
        _check(load().st_mlp_make_targets(self.handle, z_ptr, q_ptr, int(n), x_rows_ptr, r_rows_ptr))

    def loss_grad_residual(self, x_ptr: int, r_ptr: int, B: int, want_loss: bool = True, want_grads: bool = False):
        loss = ctypes.c_float()
        g = np.empty(self.n_params, np.float32) if want_grads else None
        _check(load().st_mlp_loss_grad_residual(self.handle, x_ptr, r_ptr, int(B),
                                                ctypes.byref(loss) if want_loss else None,
                                                g.ctypes.data if g is not None else None))
        return (loss.value if want_loss else None), g

    def loss_grad(self, x_ptr: int, qt_ptr: int, B: int, want_grads: bool = False):
        loss = ctypes.c_float()
        g = np.empty(self.n_params, np.float32) if want_grads else None
        _check(load().st_mlp_loss_grad(self.handle, x_ptr, qt_ptr, int(B), ctypes.byref(loss),
                                       g.ctypes.data if g is not None else None))
        return loss.value, g

    def loss_grad_async(self, x_ptr: int, qt_ptr: int, B: int):
        _check(load().st_mlp_loss_grad(self.handle, x_ptr, qt_ptr, int(B), None, None))

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        _check(load().st_mlp_adam_step(self.handle, float(lr), float(beta1), float(beta2), float(eps)))

    def train(self, x_ptr: int, r_ptr: int, n_rows: int, B: int, row_start, lr, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8, want_loss: bool = False):
        """A schedule of residual-loss Adam steps in one library call (see
        st_mlp_train): row_start and lr give each step's first row and
        learning rate.  Returns the per-step losses (or None)."""
        rs = np.ascontiguousarray(row_start, dtype=np.int64)
        lrs = np.ascontiguousarray(lr, dtype=np.float32)
        if rs.shape != lrs.shape or rs.ndim != 1:
            raise ValueError("row_start and lr must be 1-D arrays of equal length")
        losses = np.zeros(len(rs)) if want_loss else None
        _check(load().st_mlp_train(self.handle, x_ptr, r_ptr, int(n_rows), int(B), len(rs),
                                   rs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   lrs.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), float(beta1), float(beta2),
                                   float(eps),
                                   losses.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_loss else None))
        return losses

    def close(self):
        if self.handle:
            _check(load().st_mlp_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poly_term_count(degree: int) -> int:
    """Number of monomials of the 6 inputs up to the degree (1, 7, 28, 84)."""
    return [1, 7, 28, 84][int(degree)]


def poly_terms(degree: int):
    """The head polynomial's monomials in the library's order, each a tuple of
    input indices (empty for the constant)."""
    t = [()]
    if degree >= 1:
        t += [(i,) for i in range(6)]
    if degree >= 2:
        t += [(i, j) for i in range(6) for j in range(i, 6)]
    if degree >= 3:
        t += [(i, j, k) for i in range(6) for j in range(i, 6) for k in range(j, 6)]
    return t


def st_track_surrogate(ctx: int, mlp: int, n_turns: int, spin_sum_ptr: Optional[int] = None) -> None:
    _check(load().st_track_surrogate(ctx, mlp, int(n_turns), spin_sum_ptr))


def pairs_from_soa(z: np.ndarray, S: np.ndarray) -> np.ndarray:
    """[6][n] orbit + [3][n] spin -> the tracker's native 9n-double layout
    (X,Px)(Y,Py)(T,Pt)(Sx,Sy) pairs, then Sz."""
    n = z.shape[1]
    out = np.empty(9 * n, np.float64)
    for k, (a, b) in enumerate(((z[0], z[1]), (z[2], z[3]), (z[4], z[5]), (S[0], S[1]))):
        out[2 * k * n:2 * (k + 1) * n:2] = a
        out[2 * k * n + 1:2 * (k + 1) * n:2] = b
    out[8 * n:] = S[2]
    return out


def soa_from_pairs(state: np.ndarray, n: int):
    z = np.empty((6, n))
    S = np.empty((3, n))
    for k in range(3):
        z[2 * k] = state[2 * k * n:2 * (k + 1) * n:2]
        z[2 * k + 1] = state[2 * k * n + 1:2 * (k + 1) * n:2]
    S[0] = state[6 * n:8 * n:2]
    S[1] = state[6 * n + 1:8 * n:2]
    S[2] = state[8 * n:]
    return z, S


# ---- convenience object layer (still only marshalling) --------------------

class Lattice:
    def __init__(self, ring: Dict):
        self.ring = ring
        self.handle = st_lattice_create(ring["elements"], ring["G"], ring["Ggamma0"])
        self.n_elements = len(ring["elements"])

    def close(self):
        if self.handle:
            st_lattice_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tracker:
    """Tracking context for one particle ensemble on the current device."""

    def __init__(self, lattice: Lattice, n_particles: int, precision: str = "fp64", stream: Optional[int] = None):
        self.lattice = lattice
        self.n = int(n_particles)
        self.handle = st_ctx_create(lattice.handle, self.n, PRECISIONS[precision], stream)

    def set_launch(self, block_threads: int = 0, turns_per_launch: int = 0):
        st_ctx_set_launch(self.handle, block_threads, turns_per_launch)

    def upload(self, z: np.ndarray, S: np.ndarray):
        z = np.ascontiguousarray(z, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.float64)
        assert z.shape == (6, self.n) and S.shape == (3, self.n)
        st_particles_upload(self.handle, z.ctypes.data, S.ctypes.data, 0)

    def upload_device(self, z_ptr: int, s_ptr: int):
        st_particles_upload(self.handle, z_ptr, s_ptr, 1)

    def track(self, n_turns: int, spin_order: int):
        st_track(self.handle, n_turns, spin_order)

    def track_orbit(self, n_turns: int):
        st_track_orbit(self.handle, n_turns)

    def download(self):
        z = np.empty((6, self.n), np.float64)
        S = np.empty((3, self.n), np.float64)
        lost = np.empty(self.n, np.uint8)
        st_spins_download(self.handle, S.ctypes.data, z.ctypes.data, lost.ctypes.data, 0)
        return z, S, lost

    def upload_lost(self, lost: np.ndarray):
        """Restore lost flags after upload() (which clears them): with
        download() this checkpoints and resumes a run bit for bit."""
        lost = np.ascontiguousarray(lost, dtype=np.uint8)
        assert lost.shape == (self.n,)
        st_lost_upload(self.handle, lost.ctypes.data, 0)

    def download_device(self, s_ptr: int, z_ptr: Optional[int] = None, lost_ptr: Optional[int] = None):
        st_spins_download(self.handle, s_ptr, z_ptr, lost_ptr, 1)

    def close(self):
        if self.handle:
            st_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def track(ring: Dict, z: np.ndarray, S: np.ndarray, n_turns: int, spin_order: int, precision: str = "fp64",
          block_threads: int = 0, turns_per_launch: int = 0):
    """One-shot helper: host arrays in, host arrays out (z, S, lost)."""
    lat = Lattice(ring)
    tr = Tracker(lat, z.shape[1], precision)
    try:
        if block_threads or turns_per_launch:
            tr.set_launch(block_threads, turns_per_launch)
        tr.upload(z, S)
        tr.track(n_turns, spin_order)
        return tr.download()
    finally:
        tr.close()
        lat.close()
