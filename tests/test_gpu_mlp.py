"""GPU tests of the learned one-turn spin map through the C ABI: the network's
forward pass, loss gradient and Adam step against the FP64 NumPy reference
(oracle/mlp.py) with bf16 storage emulated, the tracker's one-turn quaternions
and stroboscopic sums against the CPU oracle, the FP64 linear head fit against
least squares, and the surrogate turn loop against closed forms."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1501_03450_b300 as st
import workloads as W
from oracle import mlp as M
from test_oracle_mlp import random_params

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def side_stream():
    """Every test runs on one non-default stream shared by torch's copies and
    the library calls, so that their order is the program order."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        yield s
    s.synchronize()


def cur():
    return torch.cuda.current_stream().cuda_stream


IN_SCALE = np.array([1e3, 1e4, 1e3, 1e4, 0.0, 1e3])


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).cuda()


def rand_x(B, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, 6)) * np.array([1e-3, 1e-4, 1e-3, 1e-4, 1e-2, 1e-3])


def unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def make_net(p, head, max_batch=4096):
    net = st.MLP(max_batch, cur())
    net.set_params(p.astype(np.float32))
    net.set_head(head["q0"], head["lin"], head["scale"], head["in_scale"])
    return net


def f32_params(p):
    return p.astype(np.float32).astype(np.float64)


def head_for(seed, scale=0.05, lin=True):
    rng = np.random.default_rng(seed)
    return dict(q0=unit(rng.standard_normal(4)), lin=(0.01 * rng.standard_normal((4, 6)) if lin else None),
                scale=scale, in_scale=IN_SCALE)




@pytest.mark.parametrize("B", [1, 128, 300, 2048])
def test_forward_matches_reference(B):
    """Inference against the reference with the weights and activations
    rounded to bf16 and the input split into bf16 hi + lo.  The kernels
    accumulate in FP32 and round FP32 sums to bf16, the reference rounds FP64
    sums: a rounding decision differs only where the two sums straddle a bf16
    rounding boundary (probability ~ 2^-24 sqrt(256) / 2^-8 per activation),
    which moves that activation by one bf16 step (2^-8 relative) and the next
    layer's sums by |w| 2^-8 |a|.  Rows hit by such flips differ by up to about
    one bf16 step of y (|dq| <= 1e-2 s), the average row far less; without the
    bf16 emulation every row differs by ~2^-9 |y|."""
    p = random_params(21, last_scale=1.0)
    h = head_for(3)
    x = rand_x(B, 4)
    net = make_net(p, h)
    xd = dev(x, np.float32)
    q = torch.empty((B, 4), dtype=torch.float32, device="cuda")
    net.forward(xd.data_ptr(), B, q.data_ptr())
    qg = q.cpu().numpy().astype(np.float64)        # same stream: ordered after the forward pass
    x32 = x.astype(np.float32).astype(np.float64)
    qo, _ = M.forward(f32_params(p), x32, h, bf16=True)
    qf, _ = M.forward(p, x, h, bf16=False)
    err = np.abs(qg - qo)
    assert err.max() < 1e-2 * h["scale"], err.max()
    assert err.mean() < 5e-4 * h["scale"], err.mean()
    assert np.abs(np.linalg.norm(qg, axis=1) - 1).max() < 1e-6
    if B >= 128:
        assert err.mean() < 0.2 * np.abs(qg - qf).mean()
    net.close()


# Gradient tolerance.  The reference emulates every bf16 store of the
# kernels (weights, activations, dL/dy, SiLU'(z), dL/dz) and computes in FP64; what is
# left is the kernels' FP32 accumulation: relative ~2^-24 sqrt(K) per sum (1e-5
# for K = 32768), and the bf16 stores whose FP32 and FP64 values fall on
# opposite sides of a rounding boundary.  Such a flip has probability
# ~2^-24 sqrt(256) / 2^-8 = 2^-12 per stored value and changes it by 2^-8
# relative, adding ~sqrt(2^-12) 2^-8 = 6e-5 to a block's relative L2 error
# per stored stage; thirteen stages (four activations, dL/dy, four SiLU'(z),
# four dL/dz; SiLU'(z) from the fast FP32 exponential and division, 2 ulp,
# flips less often) give ~2.2e-4.  A bias gradient is a sum over the batch of values of both signs, so
# its relative error is larger by the cancellation of that sum (measured: up
# to 7.3e-4 for b1 at a batch of 1000, 3e-5 to 3e-4 elsewhere).  The bound
# keeps a factor 3 over the largest measured block.
GRAD_REL_TOL = 2e-3


@pytest.mark.parametrize("B", [128, 1000, 10000])
def test_fused_inference_equals_layer_by_layer(B):
    """The fused five-layer inference kernel (activations in shared memory,
    accumulators in tensor memory) and one GEMM per layer compute the same
    bf16 operands, FP32 accumulation order and epilogue: identical outputs,
    for a single tile, a ragged batch and the averaging ensemble's size."""
    p = random_params(23, last_scale=1.0)
    h = head_for(6)
    x = rand_x(B, 24)
    net = make_net(p, h, max_batch=max(B, 4096))
    xd = dev(x, np.float32)
    q_f = torch.empty((B, 4), dtype=torch.float32, device="cuda")
    q_l = torch.empty((B, 4), dtype=torch.float32, device="cuda")
    net.forward(xd.data_ptr(), B, q_f.data_ptr())
    net.set_fused_inference(False)
    net.forward(xd.data_ptr(), B, q_l.data_ptr())
    net.set_fused_inference(True)
    assert torch.equal(q_f, q_l)
    qo, _ = M.forward(f32_params(p), x.astype(np.float32).astype(np.float64), h, bf16=True)
    assert np.abs(q_f.cpu().numpy() - qo).max() < 1e-2 * h["scale"]
    net.close()


def test_loss_and_gradient_match_reference():
    """Loss and all 200196 gradient entries against the reference with every
    bf16 store emulated (weights, activations, dL/dy, SiLU'(z), dL/dz) and FP64
    arithmetic: every parameter block to GRAD_REL_TOL in relative L2."""
    B = 1000
    p = random_params(7, last_scale=1.0)
    h = head_for(5)
    x = rand_x(B, 8)
    qo, _ = M.forward(f32_params(p), x.astype(np.float32).astype(np.float64), h, bf16=True)
    rng = np.random.default_rng(9)
    qt = unit(qo + 0.02 * rng.standard_normal(qo.shape))
    net = make_net(p, h)
    xd, qd = dev(x, np.float32), dev(qt, np.float32)      # held: the library reads them
    loss, g = net.loss_grad(xd.data_ptr(), qd.data_ptr(), B, want_grads=True)
    x32 = x.astype(np.float32).astype(np.float64)
    qt32 = qt.astype(np.float32).astype(np.float64)
    lo, go = M.loss_grad(f32_params(p), x32, qt32, h, bf16=True, bf16_grads=True)
    assert loss == pytest.approx(lo, rel=2e-3)
    offs = np.cumsum([0] + [r * c + r for r, c in M.LAYERS])
    rels = []
    for l, (r, c) in enumerate(M.LAYERS):
        for a, b in ((offs[l], offs[l] + r * c), (offs[l] + r * c, offs[l + 1])):
            gg, gr = g[a:b].astype(np.float64), go[a:b]
            rels.append(np.linalg.norm(gg - gr) / np.linalg.norm(gr))
    print("relative L2 error per block (W1, b1, ..., W5, b5):", ["%.1e" % v for v in rels])
    assert max(rels) < GRAD_REL_TOL, rels
    net.close()


def test_adam_steps_match_reference():
    """Two Adam steps on the kernels' own gradients against Adam in FP64."""
    B = 512
    p = random_params(17, last_scale=1.0).astype(np.float32)
    h = head_for(2)
    x = dev(rand_x(B, 1), np.float32)
    qt = dev(unit(np.random.default_rng(3).standard_normal((B, 4))), np.float32)
    net = make_net(p.astype(np.float64), h)
    pe = p.astype(np.float64)
    m = np.zeros_like(pe)
    v = np.zeros_like(pe)
    for t in (1, 2):
        _, g = net.loss_grad(x.data_ptr(), qt.data_ptr(), B, want_grads=True)
        net.adam_step(1e-3, 0.9, 0.999, 1e-8)
        pe, m, v = M.adam_step(pe, m, v, g.astype(np.float64), t, 1e-3, 0.9, 0.999, 1e-8)
        pg = net.get_params().astype(np.float64)
        np.testing.assert_allclose(pg, pe, rtol=0, atol=2e-7 * np.abs(pe).max() + 1e-9)
        pe = pg
    net.close()


def test_training_reduces_loss_on_a_smooth_map():
    """Adam on a smooth synthetic map (q0 + 0.01 sin(A x)) lowers the loss
    by more than an order of magnitude in 400 steps."""
    B = 4096
    rng = np.random.default_rng(31)
    x = rand_x(B, 30)
    A = rng.standard_normal((4, 6)) * IN_SCALE
    q0 = unit(np.array([0.1, 0.2, 0.9, 0.1]))
    qt = unit(q0 + 0.01 * np.sin(x @ A.T))
    net = st.MLP(B, cur())
    from paper_1501_03450_b300.surrogate import init_params
    net.set_params(init_params(1).astype(np.float32))
    net.set_head(q0, None, 0.01, IN_SCALE)
    xd, qd = dev(x, np.float32), dev(qt, np.float32)
    l0, _ = net.loss_grad(xd.data_ptr(), qd.data_ptr(), B)
    for k in range(400):
        net.loss_grad_async(xd.data_ptr(), qd.data_ptr(), B)
        net.adam_step(2e-3 if k < 300 else 5e-4)
    l1, _ = net.loss_grad(xd.data_ptr(), qd.data_ptr(), B)
    assert l1 < 0.05 * l0, (l0, l1)
    net.close()


@pytest.mark.parametrize("B", [700, 8192])
def test_residual_loss_and_gradient_match_reference(B):
    """As the quaternion loss, to GRAD_REL_TOL; B = 8192 runs the weight
    gradients as split-K GEMMs (64 K pieces, reduced in a fixed order)."""
    p = random_params(8, last_scale=1.0)
    x = rand_x(B, 2)
    r = np.random.default_rng(4).standard_normal((B, 4))
    net = make_net(p, head_for(1), max_batch=max(B, 4096))
    xd, rd = dev(x, np.float32), dev(r, np.float32)
    loss, g = net.loss_grad_residual(xd.data_ptr(), rd.data_ptr(), B, want_grads=True)
    x32 = x.astype(np.float32).astype(np.float64)
    r32 = r.astype(np.float32).astype(np.float64)
    lo, go = M.residual_loss_grad(f32_params(p), x32, r32, IN_SCALE, bf16=True, bf16_grads=True)
    assert loss == pytest.approx(lo, rel=2e-3)
    offs = np.cumsum([0] + [a * b + a for a, b in M.LAYERS])
    rels = []
    for l, (a, b) in enumerate(M.LAYERS):
        gg, gr = g[offs[l]:offs[l + 1]].astype(np.float64), go[offs[l]:offs[l + 1]]
        rels.append(np.linalg.norm(gg - gr) / np.linalg.norm(gr))
    print(f"B={B} relative L2 error per layer:", ["%.1e" % v for v in rels])
    assert max(rels) < GRAD_REL_TOL, rels
    net.close()


def _features(xs, degree):
    cols = []
    for t in st.poly_terms(degree):
        m = np.ones(xs.shape[1])
        for i in t:
            m = m * xs[i]
        cols.append(m)
    return np.array(cols).T


@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_fit_head_is_least_squares(degree):
    """The FP64 polynomial fit against numpy's least squares over the same
    monomials; coordinates with input scale 0 drop out; lost pairs are left
    out; the reported RMS is the residual's."""
    n = 60000
    rng = np.random.default_rng(12 + degree)
    z = rng.standard_normal((6, n)) * np.array([1e-3, 1e-4, 1e-3, 1e-4, 1e-2, 1e-3])[:, None]
    q0 = unit(rng.standard_normal(4))
    xs = z * IN_SCALE[:, None]
    q = (q0[:, None] + 1e-2 * np.sin(xs[[0, 1, 2, 3]] + xs[5]) + 1e-3 * xs[0] * xs[2] * xs[3]
         + 1e-5 * rng.standard_normal((4, n)))
    lost = np.zeros(n, np.uint8)
    lost[::7] = 1
    q[:, ::7] = 1e3                                    # garbage in lost rows
    net = st.MLP(128, cur())
    net.set_head(q0, None, 1.0, IN_SCALE)
    zd, qd, ld = dev(z, np.float64), dev(q, np.float64), dev(lost, np.uint8)
    coef, rms = net.fit_head(degree, zd.data_ptr(), qd.data_ptr(), n, ld.data_ptr())
    keep = lost == 0
    F = _features(xs[:, keep], degree)
    live = np.array([4 not in t for t in st.poly_terms(degree)])
    sol, *_ = np.linalg.lstsq(F[:, live], (q[:, keep] - q0[:, None]).T, rcond=None)
    ref = np.zeros((4, len(live)))
    ref[:, live] = sol.T
    assert np.all(coef[:, ~live] == 0.0)
    np.testing.assert_allclose(coef, ref, rtol=0, atol=1e-8 * np.abs(ref).max())
    res = (q[:, keep] - q0[:, None]) - ref @ F.T
    np.testing.assert_allclose(rms, np.sqrt(np.mean(res * res, axis=1)), rtol=1e-6)
    # the installed head: residual targets (q - q0 - P(x)) / s, and x rows
    sc = np.array([0.25, 0.5, 1e-3, 2.0])
    net.set_scale(sc)
    xr = torch.empty((n, 6), dtype=torch.float32, device="cuda")
    rr = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    net.make_targets(zd.data_ptr(), qd.data_ptr(), n, xr.data_ptr(), rr.data_ptr())
    np.testing.assert_array_equal(xr.cpu().numpy(), z.T.astype(np.float32))
    r_ref = ((q - q0[:, None] - coef @ _features(xs, degree).T) / sc[:, None]).T
    np.testing.assert_allclose(rr.cpu().numpy(), r_ref.astype(np.float32), rtol=2e-7, atol=1e-9)
    net.close()


def _oracle_turn_quats(ring, z, K):
    n = z.shape[1]
    ex = np.zeros((3, n)); ex[0] = 1.0
    ey = np.zeros((3, n)); ey[1] = 1.0
    _, Sx, _ = oracle.track(ring, z, ex, 1, K)
    _, Sy, _ = oracle.track(ring, z, ey, 1, K)
    return M.quat_from_images(Sx, Sy)


@pytest.mark.parametrize("gg", [45.5, 487.0])
def test_one_turn_quaternions_match_oracle(gg):
    """The tracker's composed one-turn quaternions against the rotation the
    oracle's tracked spins define (images of x^ and y^), up to the sign fixed
    by the reference hemisphere; spins and orbits equal those of st_track."""
    ring = W.with_spin_order(W.rhic_like_ring(gg, n_cells=12), 2)
    z, S = W.gaussian_particles(261, gg, seed=40)
    qo = _oracle_turn_quats(ring, z, 2)
    q_ref = np.array([0.3, -0.2, 0.9, 0.1])
    lat = st.Lattice(ring)
    tr = st.Tracker(lat, z.shape[1], "fp64", cur())
    tr.upload(z, S)
    q = torch.full((4, z.shape[1]), 7.0, dtype=torch.float64, device="cuda")
    st.st_track_one_turn_map(tr.handle, 2, q_ref, q.data_ptr())
    zg, Sg, lg = tr.download()
    qg = q.cpu().numpy().T
    assert np.all(qg @ q_ref >= 0.0)
    sgn = np.sign(np.sum(qg * qo, axis=1))[:, None]
    assert np.abs(qg - sgn * qo).max() < 1e-11
    z1, S1, _ = st.track(ring, z, S, 1, 2)
    np.testing.assert_array_equal(zg, z1)
    np.testing.assert_array_equal(Sg, S1)
    tr.close()
    lat.close()


def test_one_turn_quaternions_skip_lost_particles():
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    z, S = W.gaussian_particles(40, 45.5, seed=2)
    z[1, 5] = 1.5                                      # lost in the first element
    lat = st.Lattice(ring)
    tr = st.Tracker(lat, 40, "fp64", cur())
    tr.upload(z, S)
    q = torch.full((4, 40), 7.0, dtype=torch.float64, device="cuda")
    st.st_track_one_turn_map(tr.handle, 2, [1.0, 0, 0, 0], q.data_ptr())
    _, _, lost = tr.download()
    assert lost[5] == 1 and lost.sum() == 1
    q2 = torch.full((4, 40), 7.0, dtype=torch.float64, device="cuda")
    st.st_track_one_turn_map(tr.handle, 2, [1.0, 0, 0, 0], q2.data_ptr())
    torch.cuda.synchronize()
    assert np.all(q2.cpu().numpy()[:, 5] == 7.0)       # already lost: untouched
    tr.close()
    lat.close()


def test_stroboscopic_sum_matches_oracle():
    """st_track_average: the spin at s = 0 summed after every turn, against
    the oracle tracked turn by turn."""
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    z, S = W.gaussian_particles(100, 45.5, seed=6)
    S = W.cap_spins(100, 0.3, seed=6)
    turns = 12
    zo, So = z.copy(), S.copy()
    acc = np.zeros_like(S)
    for _ in range(turns):
        zo, So, _ = oracle.track(ring, zo, So, 1, 2)
        acc += So
    lat = st.Lattice(ring)
    tr = st.Tracker(lat, 100, "fp64", cur())
    tr.set_launch(0, 5)                                # several turns per launch
    tr.upload(z, S)
    ssum = torch.zeros((3, 100), dtype=torch.float64, device="cuda")
    st.st_track_average(tr.handle, turns, 2, ssum.data_ptr())
    zg, Sg, _ = tr.download()
    assert np.abs(ssum.cpu().numpy() - acc).max() < 1e-11 * turns
    assert np.abs(Sg - So).max() < 1e-11 and np.abs(zg - zo).max() < 1e-11
    tr.close()
    lat.close()


def test_surrogate_with_zero_network_is_the_closed_form():
    """With zero weights and no linear term the learned map is the constant
    rotation q0: S_t = R(q0)^t S_0 for every particle, the orbit is the
    orbit-only tracker's, and the stroboscopic sum is the sum of the S_t."""
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    n, turns = 300, 25
    z, S = W.gaussian_particles(n, 45.5, seed=8)
    S = W.cap_spins(n, 0.4, seed=8)
    th = 0.7
    axis = unit(np.array([0.2, 1.0, -0.3]))
    q0 = np.array([math.cos(th / 2), *(axis * math.sin(th / 2))])
    net = st.MLP(512, cur())
    net.set_params(np.zeros(net.n_params, np.float32))
    net.set_head(q0, None, 1.0, IN_SCALE)
    lat = st.Lattice(ring)
    tr = st.Tracker(lat, n, "fp64", cur())
    tr.upload(z, S)
    ssum = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    st.st_track_surrogate(tr.handle, net.handle, turns, ssum.data_ptr())
    zg, Sg, lg = tr.download()
    qf = unit(q0)                                      # the head is FP64
    Se = S.copy()
    acc = np.zeros_like(S)
    for _ in range(turns):
        Se = M.rotate(np.tile(qf, (n, 1)), Se)
        acc += Se
    assert np.abs(Sg - Se).max() < 1e-12 * turns
    assert np.abs(ssum.cpu().numpy() - acc).max() < 1e-12 * turns * turns
    tr2 = st.Tracker(lat, n, "fp64", cur())
    tr2.upload(z, S)
    tr2.track_orbit(turns)
    z2, S2, l2 = tr2.download()
    np.testing.assert_array_equal(zg, z2)
    np.testing.assert_array_equal(S2, S)               # orbit-only leaves spins alone
    tr.close()
    tr2.close()
    lat.close()
    net.close()


def test_train_schedule_replayed_from_a_graph_equals_eager_steps():
    """st_mlp_train runs its first step eagerly and replays the others from a
    captured CUDA graph (the rows and the Adam schedule read on the device):
    after a 7-step schedule the parameters and the per-step losses equal
    those of 7 one-step calls, which all run eagerly, bit for bit."""
    B, n_rows = 1000, 5000
    rng = np.random.default_rng(77)
    x = rand_x(n_rows, 40)
    r = rng.standard_normal((n_rows, 4)) * 0.1
    p = random_params(9, last_scale=1.0)
    xd, rd = dev(x, np.float32), dev(r, np.float32)
    rows = np.array([0, 1200, 4000, 300, 2500, 3999, 17], dtype=np.int64)
    lrs = np.array([2e-3, 2e-3, 1e-3, 1e-3, 5e-4, 5e-4, 5e-4], dtype=np.float32)
    a = make_net(p, head_for(1), max_batch=B)
    la = a.train(xd.data_ptr(), rd.data_ptr(), n_rows, B, rows, lrs, want_loss=True)
    pa = a.get_params()
    b = make_net(p, head_for(1), max_batch=B)
    lb = [b.train(xd.data_ptr(), rd.data_ptr(), n_rows, B, rows[k:k + 1], lrs[k:k + 1], want_loss=True)[0]
          for k in range(len(rows))]
    pb = b.get_params()
    a.close()
    b.close()
    assert np.array_equal(pa, pb)
    assert np.allclose(la, lb, rtol=1e-12, atol=0.0)   # the loss is an atomic sum: order may vary
    assert not np.array_equal(pa, p.astype(np.float32))
