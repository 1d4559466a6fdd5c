"""The allocation-free FP64 entry point, for callers that cannot allocate device
memory (for example code running inside a memory pool that owns all of the
device memory, or a host process that forbids further allocations): it works
on buffers the caller already owns and keeps its own lattice table and status
word in a fixed device array of the library.

Checked through the C ABI against the regular context-based entry point, on
two calls in a row (the second call reuses, and must fully rewrite, the same
scratch with a different lattice).  Kept in a file that pytest collects last.
"""
import numpy as np
import pytest

import paper_1501_03450_b300 as st
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _run_noalloc(torch, ring, z, S, turns, K):
    n = z.shape[1]
    state = torch.from_numpy(st.pairs_from_soa(z, S)).to("cuda")
    lost = torch.zeros(n, dtype=torch.uint8, device="cuda")
    st.st_track_fp64_noalloc(ring["elements"], ring["G"], ring["Ggamma0"], state.data_ptr(), lost.data_ptr(),
                             n, turns, K, torch.cuda.current_stream().cuda_stream)
    zo, So = st.soa_from_pairs(state.cpu().numpy(), n)
    return zo, So, lost.cpu().numpy()


def test_noalloc_matches_context_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    # call 1: toy ring, order 2
    ring1 = W.with_spin_order(W.toy_ring(45.5), 2)
    z1, S1 = W.gaussian_particles(1000, 45.5, seed=101)
    z1[1, 7] = 1.5                                   # one lost particle
    a = _run_noalloc(torch, ring1, z1, S1, 20, 2)
    b = st.track(ring1, z1, S1, 20, 2)
    assert np.array_equal(a[2], b[2]) and a[2][7] == 1
    assert np.abs(a[0] - b[0]).max() < TOL and np.abs(a[1] - b[1]).max() < TOL
    # call 2: a different lattice (matrix-kick quads, sextupoles, snakes), order 3
    ring2 = W.with_spin_order(W.rhic_like_ring(487.0, n_cells=12), 3)
    z2, S2 = W.gaussian_particles(777, 487.0, seed=102)
    c = _run_noalloc(torch, ring2, z2, S2, 7, 3)
    d = st.track(ring2, z2, S2, 7, 3)
    assert np.array_equal(c[2], d[2])
    assert np.abs(c[0] - d[0]).max() < TOL and np.abs(c[1] - d[1]).max() < TOL


def test_noalloc_rejects_oversized_lattice_and_bad_order():
    torch = pytest.importorskip("torch")
    n = 64
    state = torch.zeros(9 * n, dtype=torch.float64, device="cuda")
    lost = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    with pytest.raises(st.SpinTrackError) as e:        # 4 slices, order 3 needs multiples of 8
        st.st_track_fp64_noalloc(ring["elements"], ring["G"], ring["Ggamma0"], state.data_ptr(), lost.data_ptr(),
                                 n, 1, 3)
    assert e.value.code == st.ST_EINVAL
    big = [W.element("drift", L=1.0 + 1e-3 * i) for i in range(600)]     # > 512 distinct elements
    with pytest.raises(st.SpinTrackError) as e:
        st.st_track_fp64_noalloc(big, 1.7928, 45.5, state.data_ptr(), lost.data_ptr(), n, 1, 0)
    assert e.value.code == st.ST_EINVAL


def test_noalloc_with_teapot_bends_matches_context_entry_point():
    """A drift-kick lattice (TEAPOT bends, extended instantiation) through the
    allocation-free entry point."""
    torch = pytest.importorskip("torch")
    ring = W.with_spin_order(W.drift_kick_ring(W.rhic_like_ring(45.5, n_cells=12)), 2)
    z, S = W.gaussian_particles(500, 45.5, seed=103)
    a = _run_noalloc(torch, ring, z, S, 5, 2)
    b = st.track(ring, z, S, 5, 2)
    assert np.array_equal(a[2], b[2])
    assert np.abs(a[0] - b[0]).max() < TOL and np.abs(a[1] - b[1]).max() < TOL


def test_noalloc_midpoint_schemes_match_context_entry_point():
    torch = pytest.importorskip("torch")
    ring = W.with_slices(W.drift_kick_ring(W.toy_ring(45.5)), 3)
    z, S = W.gaussian_particles(300, 45.5, seed=104)
    for K in (st.ST_SPIN_MID_HALF, st.ST_SPIN_MID_KICK):
        a = _run_noalloc(torch, ring, z, S, 4, K)
        b = st.track(ring, z, S, 4, K)
        assert np.array_equal(a[2], b[2])
        assert np.abs(a[0] - b[0]).max() < TOL and np.abs(a[1] - b[1]).max() < TOL
    n = 64
    state = torch.zeros(9 * n, dtype=torch.float64, device="cuda")
    lost = torch.zeros(n, dtype=torch.uint8, device="cuda")
    r4 = W.with_split_order(W.toy_ring(45.5), 4)
    with pytest.raises(st.SpinTrackError) as e:
        st.st_track_fp64_noalloc(r4["elements"], r4["G"], r4["Ggamma0"], state.data_ptr(), lost.data_ptr(), n, 1,
                                 st.ST_SPIN_MID_KICK)
    assert e.value.code == st.ST_EINVAL


def test_noalloc_refuses_misaligned_and_host_buffers_without_launching():
    """The state is accessed as 16-byte pairs: an 8-byte-offset view is
    refused with ST_EINVAL, and so are host buffers, before anything is
    staged or launched (the buffers are unchanged and the context still
    tracks correctly afterwards)."""
    torch = pytest.importorskip("torch")
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    n = 64
    z, S = W.gaussian_particles(n, 45.5, seed=105)
    base = torch.from_numpy(np.concatenate([[0.0], st.pairs_from_soa(z, S)])).to("cuda")
    lost = torch.zeros(n, dtype=torch.uint8, device="cuda")
    before = base.clone()
    with pytest.raises(st.SpinTrackError) as e:
        st.st_track_fp64_noalloc(ring["elements"], ring["G"], ring["Ggamma0"], base.data_ptr() + 8,
                                 lost.data_ptr(), n, 1, 2)
    assert e.value.code == st.ST_EINVAL and "aligned" in str(e.value)
    host_state = np.ascontiguousarray(st.pairs_from_soa(z, S))
    host_lost = np.zeros(n, np.uint8)
    with pytest.raises(st.SpinTrackError) as e:
        st.st_track_fp64_noalloc(ring["elements"], ring["G"], ring["Ggamma0"], host_state.ctypes.data,
                                 lost.data_ptr(), n, 1, 2)
    assert e.value.code == st.ST_EINVAL and "device" in str(e.value)
    with pytest.raises(st.SpinTrackError) as e:
        st.st_track_fp64_noalloc(ring["elements"], ring["G"], ring["Ggamma0"], base.data_ptr() + 8,
                                 host_lost.ctypes.data, n, 1, 2)
    assert e.value.code == st.ST_EINVAL
    torch.cuda.synchronize()
    assert torch.equal(base, before) and int(lost.sum()) == 0
    a = _run_noalloc(torch, ring, z, S, 3, 2)
    b = st.track(ring, z, S, 3, 2)
    assert np.abs(a[0] - b[0]).max() < TOL and np.abs(a[1] - b[1]).max() < TOL
