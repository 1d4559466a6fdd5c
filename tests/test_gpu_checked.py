"""The index-checked build (the same sources compiled with -DST_CHECKED: every
element-table index and batch work item is tested before use, a violation
writes a status word instead of reading out of range) runs the trackers
without reporting a violation and gives the oracle's results.  It is loaded
through SPINTRACK_LIB in a child process, as a user would select it."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import workloads as W
from paper_1501_03450_b300 import _build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import paper_1501_03450_b300 as st
import workloads as W
assert st.LIB_PATH.endswith("libspintrack_checked.so"), st.LIB_PATH
out = {}
toy = W.with_spin_order(W.toy_ring(45.5), 2)
z, S = W.gaussian_particles(300, 45.5, seed=5)
z[1, 7] = 1.5
out["fp64_z"], out["fp64_S"], out["fp64_l"] = st.track(toy, z, S, 20, 2)
ext = W.with_fringes(W.with_split_order(W.rbend_ring(45.5), 4))
ext = W.with_spin_order(ext, 2)
ext["elements"] += [W.element("solenoid", L=2.0, n_slices=4, k1=0.05)]
out["ext_z"], out["ext_S"], out["ext_l"] = st.track(ext, z, S, 5, 2)
out["mix_z"], out["mix_S"], out["mix_l"] = st.track(toy, z, S, 20, 2, precision="mixed")
dk = W.drift_kick_ring(W.with_fringes(W.toy_ring(45.5)))
out["mid_z"], out["mid_S"], out["mid_l"] = st.track(dk, z, S, 5, st.ST_SPIN_MID_KICK)
dk2 = W.with_spin_order(dk, 2)
out["mdk_z"], out["mdk_S"], out["mdk_l"] = st.track(dk2, z, S, 5, 2, precision="mixed")
out["mdm_z"], out["mdm_S"], out["mdm_l"] = st.track(dk, z, S, 5, st.ST_SPIN_MID_HALF, precision="mixed")
sol = W.with_spin_order(W.solenoid_ring(45.5), 2)
out["msol_z"], out["msol_S"], out["msol_l"] = st.track(sol, z, S, 3, 2, precision="mixed")
b = st.Batch([toy, W.with_spin_order(W.rhic_like_ring(300.0, n_cells=6), 2)], [300, 77], "mixed")
b.upload(0, z, S)
z2, S2 = W.gaussian_particles(77, 300.0, seed=6)
b.upload(1, z2, S2)
b.track(3, 2)
out["bat_z"], out["bat_S"], out["bat_l"] = b.download(1)
b.close()
np.savez(sys.argv[1], **out)
"""


def test_checked_build_runs_clean_and_matches_the_oracle(tmp_path):
    if not _build.up_to_date(checked=True):
        _build.build(checked=True)
    out = tmp_path / "checked.npz"
    env = dict(os.environ, SPINTRACK_LIB=_build.LIB_CHECKED, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD, str(out)], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    d = np.load(out)
    toy = W.with_spin_order(W.toy_ring(45.5), 2)
    z, S = W.gaussian_particles(300, 45.5, seed=5)
    z[1, 7] = 1.5
    zo, So, lo = oracle.track(toy, z, S, 20, 2)
    assert np.array_equal(d["fp64_l"], lo) and lo[7] == 1
    assert np.abs(d["fp64_z"] - zo).max() < 1e-11 and np.abs(d["fp64_S"] - So).max() < 1e-11
    ext = W.with_fringes(W.with_split_order(W.rbend_ring(45.5), 4))
    ext = W.with_spin_order(ext, 2)
    ext["elements"] += [W.element("solenoid", L=2.0, n_slices=4, k1=0.05)]
    zo, So, lo = oracle.track(ext, z, S, 5, 2)
    assert np.array_equal(d["ext_l"], lo)
    assert np.abs(d["ext_z"] - zo).max() < 1e-11 and np.abs(d["ext_S"] - So).max() < 1e-11
    dk = W.drift_kick_ring(W.with_fringes(W.toy_ring(45.5)))
    zo, So, lo = oracle.track(dk, z, S, 5, oracle.MID_KICK)
    assert np.array_equal(d["mid_l"], lo)
    assert np.abs(d["mid_z"] - zo).max() < 1e-11 and np.abs(d["mid_S"] - So).max() < 1e-11
    # mixed precision: its own accuracy against the FP64 oracle on this ring
    zo, So, lo = oracle.track(toy, z, S, 20, 2)
    assert np.array_equal(d["mix_l"], lo)
    assert np.abs(d["mix_S"] - So).max() < 1e-6
    z2, S2 = W.gaussian_particles(77, 300.0, seed=6)
    zo, So, lo = oracle.track(W.with_spin_order(W.rhic_like_ring(300.0, n_cells=6), 2), z2, S2, 3, 2)
    assert np.array_equal(d["bat_l"], lo)
    assert np.abs(d["bat_S"] - So).max() < 1e-6
    # the mixed tracker's TEAPOT instantiation (Romberg and midpoint kernels)
    for key, ring, K in (("mdk", W.with_spin_order(dk, 2), 2), ("mdm", dk, oracle.MID_HALF),
                         ("msol", W.with_spin_order(W.solenoid_ring(45.5), 2), 2)):
        zo, So, lo = oracle.track(ring, z, S, 3 if key == "msol" else 5, K)
        assert np.array_equal(d[key + "_l"], lo)
        assert np.abs(d[key + "_S"] - So).max() < 1e-6
