"""Build the spintrack shared library in-tree with nvcc for sm_103a.

Every `.cu` file is compiled to its own object in parallel (no device symbol
crosses a file, so no relocatable device code is needed), then the objects
are linked into the shared library.  Objects live under `_build/` and are
rebuilt when their source or any header is newer.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libspintrack.so")
# checked build: the same sources with -DST_CHECKED (index tests that record a
# status instead of reading out of range); selected with SPINTRACK_LIB
LIB_CHECKED = os.path.join(PKG, "libspintrack_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC",
    "-I", INCLUDE, "-I", CSRC,
]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(INCLUDE, "spintrack.h")]


def deps():
    return sources() + headers()


def _newest_header() -> float:
    return max(os.path.getmtime(h) for h in headers())


def up_to_date(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in deps())


def _obj_path(src: str, checked: bool) -> str:
    base = os.path.splitext(os.path.basename(src))[0]
    return os.path.join(OBJ, base + ("_checked" if checked else "") + ".o")


def _compile(nvcc: str, src: str, obj: str, checked: bool, verbose: bool):
    cmd = ([nvcc] + NVCC_FLAGS + (["-DST_CHECKED"] if checked else []) + (["-Xptxas", "-v"] if verbose else [])
           + ["-c", src, "-o", obj + ".tmp"])
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode == 0:
        os.replace(obj + ".tmp", obj)
    return src, res


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(checked):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ, exist_ok=True)
    newest_h = _newest_header()
    todo = []
    for src in sources():
        obj = _obj_path(src, checked)
        if (force or verbose or not os.path.exists(obj)
                or os.path.getmtime(obj) < max(os.path.getmtime(src), newest_h)):
            todo.append((src, obj))
    jobs = max(1, min(len(todo), os.cpu_count() or 1))
    failed = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for src, res in ex.map(lambda so: _compile(nvcc, so[0], so[1], checked, verbose), todo):
            if res.returncode != 0:
                failed.append(src)
                sys.stderr.write(res.stdout + res.stderr)
            elif verbose:
                sys.stderr.write(res.stderr)
    if failed:
        raise RuntimeError(f"nvcc failed on {', '.join(os.path.basename(f) for f in failed)}")
    objs = [_obj_path(src, checked) for src in sources()]
    cmd = [nvcc] + ARCH + ["-shared", "-Xcompiler", "-fPIC"] + objs + ["-o", lib + ".tmp"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError(f"nvcc failed linking {os.path.basename(lib)}")
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
