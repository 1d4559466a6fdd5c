"""Host-side checks of the C ABI (no GPU needed): the shared library builds,
loads, and exports every function include/spintrack.h declares; argument
validation that happens before any CUDA call."""
import ctypes
import os
import re

import pytest

import paper_1501_03450_b300 as st

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(inc, fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(st_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("st_lattice_create", "st_particles_upload", "st_track", "st_spins_download"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = st.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in st.SIGNATURES, f"binding lacks a signature for {name}"


def test_checked_build_exports_the_same_symbols():
    """The index-checked build (same sources, -DST_CHECKED) is a drop-in
    replacement selected with SPINTRACK_LIB."""
    from paper_1501_03450_b300 import _build
    if not os.path.exists(_build.LIB_CHECKED) or not _build.up_to_date(checked=True):
        _build.build(checked=True)
    lib = ctypes.CDLL(_build.LIB_CHECKED)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_error_string():
    lib = st.load()
    assert b"sm_103a" in lib.st_version()
    assert isinstance(lib.st_last_error(), bytes)


def test_lattice_validation_happens_on_host():
    lib = st.load()
    out = ctypes.c_void_p()
    ref = st.StReference(1.7928, 45.5)
    # n < 1
    assert lib.st_lattice_create(None, 0, ctypes.byref(ref), ctypes.byref(out)) == st.ST_EINVAL
    # unknown type
    arr = st.elements_array([dict(type="drift", L=1.0, n_slices=1, k1=0, k2=0, angle=0, eta=1,
                                  snake_phi=0, snake_mu=0)])
    arr[0].type = 9
    assert lib.st_lattice_create(arr, 1, ctypes.byref(ref), ctypes.byref(out)) == st.ST_EINVAL
    assert b"unknown type" in lib.st_last_error()
    # bend with zero angle
    arr = st.elements_array([dict(type="sbend", L=1.0, n_slices=4, k1=0, k2=0, angle=0.0, eta=1,
                                  snake_phi=0, snake_mu=0)])
    assert lib.st_lattice_create(arr, 1, ctypes.byref(ref), ctypes.byref(out)) == st.ST_EINVAL
    # gamma0 <= 1
    bad = st.StReference(1.7928, 1.0)
    arr = st.elements_array([dict(type="drift", L=1.0, n_slices=1, k1=0, k2=0, angle=0, eta=1,
                                  snake_phi=0, snake_mu=0)])
    assert lib.st_lattice_create(arr, 1, ctypes.byref(bad), ctypes.byref(out)) == st.ST_EINVAL
    assert out.value is None


def test_null_context_calls_are_rejected():
    lib = st.load()
    assert lib.st_track(None, 1, 2) == st.ST_EINVAL
    assert lib.st_particles_upload(None, None, None, 0) == st.ST_EINVAL
    assert lib.st_spins_download(None, None, None, None, 0) == st.ST_EINVAL
    assert lib.st_ctx_set_launch(None, 64, 1) == st.ST_EINVAL
    assert lib.st_ctx_destroy(None) == st.ST_OK
    assert lib.st_lattice_destroy(None) == st.ST_OK


def header_constants():
    txt = open(os.path.join(ROOT, "include", "spintrack.h")).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define\s+(ST_\w+)\s+(-?\d+)", txt, flags=re.M)}


def test_binding_constants_match_the_header():
    consts = header_constants()
    for name, value in consts.items():
        assert getattr(st, name) == value, name
    assert st.TYPE_CODES["teapot"] == consts["ST_TEAPOT"]
    assert (consts["ST_SPIN_MID_HALF"], consts["ST_SPIN_MID_KICK"]) == (-1, -2)


def test_teapot_validation_happens_on_host():
    """Invalid TEAPOT bends are rejected before any device call; the fourth-
    order split is allowed for them (and still refused for an exact bend)."""
    lib = st.load()
    out = ctypes.c_void_p()
    ref = st.StReference(1.7928, 45.5)
    base = dict(type="teapot", L=3.0, n_slices=4, k1=0, k2=0, angle=0.1, eta=1, snake_phi=0, snake_mu=0)
    for bad in (dict(angle=0.0), dict(angle=4.5), dict(L=0.0), dict(split_order=3), dict(fringe=2)):
        arr = st.elements_array([dict(base, **bad)])
        assert lib.st_lattice_create(arr, 1, ctypes.byref(ref), ctypes.byref(out)) == st.ST_EINVAL, bad
    arr = st.elements_array([dict(base, type="sbend", split_order=4)])
    assert lib.st_lattice_create(arr, 1, ctypes.byref(ref), ctypes.byref(out)) == st.ST_EINVAL
    assert b"split_order" in lib.st_last_error()
    assert out.value is None


def test_tuner_and_midpoint_argument_checks_happen_on_host():
    """st_tune_slicing rejects null outputs, empty input, a non-positive bound
    and invalid elements before any device call."""
    lib = st.load()
    ref = st.StReference(1.7928, 45.5)
    arr = st.elements_array([dict(type="mult", L=1.0, n_slices=4, k1=0.1, k2=0, angle=0, eta=1, snake_phi=0,
                                  snake_mu=0)])
    z = (ctypes.c_double * 6)()
    s = (ctypes.c_double * 3)()
    nb, K = ctypes.c_int32(), ctypes.c_int32()
    args = lambda bound, n=1, nbp=ctypes.byref(nb): (arr, n, ctypes.byref(ref), z, s, 1, bound, nbp, ctypes.byref(K),
                                                     None, None, None, None)
    assert lib.st_tune_slicing(*args(0.0)) == st.ST_EINVAL
    assert lib.st_tune_slicing(*args(1e-6, n=0)) == st.ST_EINVAL
    assert lib.st_tune_slicing(*args(1e-6, nbp=None)) == st.ST_EINVAL
    bad = st.elements_array([dict(type="thin_mult", L=0.5, n_slices=4, k1=0.1, k2=0, angle=0, eta=1, snake_phi=0,
                                  snake_mu=0)])
    assert lib.st_tune_slicing(bad, 1, ctypes.byref(ref), z, s, 1, 1e-6, ctypes.byref(nb), ctypes.byref(K),
                               None, None, None, None) == st.ST_EINVAL
    assert b"thin lens" in lib.st_last_error()
    # the midpoint schemes on a null context are rejected like any order
    assert lib.st_track(None, 1, st.ST_SPIN_MID_KICK) == st.ST_EINVAL


def test_particle_count_limit_is_checked_before_any_device_call():
    """The kernels index particles with a 32-bit int, so a context holds at
    most 2^31 - 1 particles; 2^31 is refused before the lattice handle is
    touched or any memory is allocated (the handle here is a dummy that the
    call must not dereference), and so is 2^31 for the allocation-free entry
    point."""
    lib = st.load()
    dummy = ctypes.create_string_buffer(8)
    out = ctypes.c_void_p()
    assert lib.st_ctx_create(ctypes.addressof(dummy), 1 << 31, st.ST_FP64, None, ctypes.byref(out)) == st.ST_EINVAL
    assert b"2^31 - 1" in lib.st_last_error()
    assert out.value is None
    ref = st.StReference(1.7928, 45.5)
    arr = st.elements_array([dict(type="drift", L=1.0, n_slices=1, k1=0, k2=0, angle=0, eta=1, snake_phi=0,
                                  snake_mu=0)])
    assert lib.st_track_fp64_noalloc(arr, 1, ctypes.byref(ref), ctypes.addressof(dummy), ctypes.addressof(dummy),
                                     1 << 31, 1, 0, None) == st.ST_EINVAL
