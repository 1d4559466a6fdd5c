"""GPU parity: the CUDA tracker through the C ABI against the CPU oracle on the
same seeded inputs, element by element (every coordinate and spin component
of every particle).  Tolerance 1e-11 absolute on the canonical coordinates
(X, Y, T in m; Px, Py, Pt scaled by p0) and on the spin components."""
import math

import numpy as np
import pytest

import oracle
import paper_1501_03450_b300 as st
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-11


def compare(ring, z, S, turns, K, tol=TOL, **launch):
    zg, Sg, lg = st.track(ring, z, S, turns, K, **launch)
    zo, So, lo = oracle.track(ring, z, S, turns, K)
    assert np.array_equal(lg, lo)
    dz = np.abs(zg - zo).max(axis=1)
    ds = np.abs(Sg - So).max()
    assert dz.max() < tol and ds < tol, (dz, ds)
    return dz, ds


def test_toy_ring_100_turns_full_parity():
    """Toy proton ring, 1024 Gaussian particles, Romberg order 2, 100 turns."""
    w = W.workload("toy_ring_1024")
    z, S = W.gaussian_particles(w["n_particles"], 45.5, seed=w["seed"])
    compare(w["ring"], z, S, w["turns"], 2)


@pytest.mark.parametrize("K", [0, 1, 2, 3, 4])
def test_toy_ring_every_romberg_order(K):
    ring = W.with_spin_order(W.toy_ring(45.5), K)
    z, S = W.gaussian_particles(333, 45.5, seed=11 + K)      # ragged tail of blocks
    compare(ring, z, S, 10, K)


@pytest.mark.parametrize("gg", [45.5, 487.0])
@pytest.mark.parametrize("K", [2, 3])
def test_rhic_like_ring_matrix_kick_sextupoles_snakes(gg, K):
    ring = W.with_spin_order(W.rhic_like_ring(gg, n_cells=20), K)
    z, S = W.gaussian_particles(300, gg, seed=5)
    compare(ring, z, S, 10, K)


def test_full_size_rhic_ring_sampled():
    """The bench workload's full size (10^5 particles, 108-cell ring, order 2)
    in the bench's launch shape; 200 particles sampled across the ensemble are
    tracked by the oracle and compared."""
    w = W.workload("rhic_like_1e5")
    z, S = W.gaussian_particles(w["n_particles"], 45.5, seed=w["seed"])
    turns = 3
    zg, Sg, lg = st.track(w["ring"], z, S, turns, 2)
    idx = np.linspace(0, w["n_particles"] - 1, 200).astype(int)
    zo, So, lo = oracle.track(w["ring"], z[:, idx], S[:, idx], turns, 2)
    assert np.array_equal(lg[idx], lo)
    assert np.abs(zg[:, idx] - zo).max() < TOL
    assert np.abs(Sg[:, idx] - So).max() < TOL
    assert lg.sum() == 0
    assert np.abs(np.linalg.norm(Sg, axis=0) - 1).max() < 1e-12


def test_edge_cases_tiny_on_axis_and_lost():
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    # a single particle on axis: Omega vanishes in the quadrupoles (zero-angle edge rotations)
    z = np.zeros((6, 1)); S = np.array([[0.0], [0.0], [1.0]])
    compare(ring, z, S, 5, 2)
    # 33 particles (one full warp + 1), one of them lost in the first element
    z, S = W.gaussian_particles(33, 45.5, seed=3)
    z[1, 17] = 1.5
    zg, Sg, lg = st.track(ring, z, S, 4, 2)
    zo, So, lo = oracle.track(ring, z, S, 4, 2)
    assert lg[17] == 1 and lo[17] == 1 and lg.sum() == 1
    assert np.abs(zg - zo).max() < TOL and np.abs(Sg - So).max() < TOL


def test_launch_shapes_give_identical_results():
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    z, S = W.gaussian_particles(200, 45.5, seed=9)
    a = st.track(ring, z, S, 6, 2, block_threads=32, turns_per_launch=1)
    b = st.track(ring, z, S, 6, 2, block_threads=128, turns_per_launch=6)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_zero_turns_and_bad_orders():
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    z, S = W.gaussian_particles(40, 45.5, seed=2)
    zg, Sg, lg = st.track(ring, z, S, 0, 2)
    assert np.array_equal(zg, z) and np.array_equal(Sg, S)
    lat = st.Lattice(ring)
    tr = st.Tracker(lat, 40)
    with pytest.raises(st.SpinTrackError) as e:
        tr.track(1, 2)                          # before upload
    assert e.value.code == st.ST_ESTATE
    tr.upload(z, S)
    with pytest.raises(st.SpinTrackError) as e:
        tr.track(1, 3)                          # 4 slices not divisible by 8
    assert e.value.code == st.ST_EINVAL
    with pytest.raises(st.SpinTrackError):
        tr.track(-1, 2)
    tr.close()
    lat.close()


def test_device_pointers_and_torch_stream():
    torch = pytest.importorskip("torch")
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    z, S = W.gaussian_particles(256, 45.5, seed=4)
    dev = torch.device("cuda:0")
    zt = torch.from_numpy(z).to(dev)
    St = torch.from_numpy(S).to(dev)
    stream = torch.cuda.Stream()
    lat = st.Lattice(ring)
    tr = st.Tracker(lat, 256, stream=stream.cuda_stream)
    tr.upload_device(zt.data_ptr(), St.data_ptr())
    tr.track(5, 2)
    So = torch.empty_like(St)
    zo = torch.empty_like(zt)
    tr.download_device(So.data_ptr(), zo.data_ptr())
    zr, Sr, _ = oracle.track(ring, z, S, 5, 2)
    assert np.abs(zo.cpu().numpy() - zr).max() < TOL
    assert np.abs(So.cpu().numpy() - Sr).max() < TOL
    tr.close()
    lat.close()


@pytest.mark.parametrize("gg", [1.9, 10.0, 45.5, 150.0, 487.0, 2000.0])
def test_edge_rotation_angle_sweep(gg):
    """Edge rotations from 0.05 rad to 200 rad per slice (every branch of the
    edge-quaternion series, including halving and squaring back) against the
    oracle's library sin/cos; on-axis also against the closed form."""
    el = W.element("sbend", L=3.0, n_slices=4, angle=0.4)
    ring = W.single_element_ring(el, gg)
    z, S = W.gaussian_particles(64, gg, seed=21, sigmas=dict(x=5e-3, px=5e-4))
    z[:, 0] = 0.0
    S = W.cap_spins(64, math.pi, seed=22)
    zg, Sg, _ = st.track(ring, z, S, 1, 2)
    zo, So, _ = oracle.track(ring, z, S, 1, 2)
    tol = 1e-15 * (20 + gg * 0.4)
    assert np.abs(Sg - So).max() < tol
    assert np.abs(zg - zo).max() < 1e-13
    a = -gg * 0.4                    # on axis: rotation by -G gamma theta about y
    s0 = S[:, 0]
    exp = np.array([s0[0] * math.cos(a) + s0[2] * math.sin(a), s0[1], -s0[0] * math.sin(a) + s0[2] * math.cos(a)])
    assert np.abs(Sg[:, 0] - exp).max() < tol


def test_strong_bend_large_deflections():
    """Large transverse momenta in a strongly bending magnet exercise the
    library-asin branch of the bend's angle difference."""
    el = W.element("sbend", L=1.0, n_slices=8, angle=1.2, eta=1.05)
    ring = W.with_spin_order(W.single_element_ring(el, 45.5), 3)
    z, S = W.gaussian_particles(128, 45.5, seed=8, sigmas=dict(x=0.05, px=0.08, y=0.01, py=0.02, delta=0.02))
    compare(ring, z, S, 1, 3, tol=1e-12)
