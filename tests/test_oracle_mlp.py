"""Pins of the FP64 reference of the learned one-turn spin map (oracle/mlp.py)
against facts that do not come from it: central finite differences of its own
loss (gradient), library routines (torch's bfloat16 cast, scipy's logistic
function), Rodrigues' rotation formula, closed forms of Adam's first step and
of a network with zero weights."""
import math

import numpy as np
import pytest
import torch
from scipy.special import expit

from oracle import mlp as M

HEAD = dict(q0=np.array([0.05, 0.1, 0.99, -0.02]), lin=None, scale=0.3,
            in_scale=np.array([1e3, 1e4, 1e3, 1e4, 0.0, 1e3]))


def _inputs(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, 6)) * np.array([1e-3, 1e-4, 1e-3, 1e-4, 1e-2, 1e-3])
    qt = rng.standard_normal((B, 4))
    qt /= np.linalg.norm(qt, axis=1, keepdims=True)
    return x, qt


def random_params(seed, last_scale=1.0):
    """Random network weights (He-normal), biases small random."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (r, c) in enumerate(M.LAYERS):
        parts.append(rng.standard_normal(r * c) * np.sqrt(2.0 / c) * (last_scale if l == 4 else 1.0))
        parts.append(0.01 * rng.standard_normal(r))
    return np.concatenate(parts)


def test_param_layout():
    assert M.param_count() == 6 * 256 + 256 + 3 * (256 * 256 + 256) + 4 * 256 + 4 == 200196
    p = np.arange(M.param_count(), dtype=np.float64)
    layers = M.unpack(p)
    assert layers[0][0].shape == (256, 6) and layers[0][0][0, 1] == 1.0
    assert layers[0][1][0] == 1536.0
    assert layers[4][0].shape == (4, 256) and layers[4][1][-1] == M.param_count() - 1


def test_round_bf16_ties_and_library_cast():
    u = 2.0 ** -7                                    # bf16 spacing at 1
    assert M.round_bf16(np.array([1.0]))[0] == 1.0
    assert M.round_bf16(np.array([1.0 + u / 2]))[0] == 1.0             # tie -> even
    assert M.round_bf16(np.array([1.0 + 1.5 * u]))[0] == 1.0 + 2 * u   # tie -> even
    assert M.round_bf16(np.array([1.0 + 0.51 * u]))[0] == 1.0 + u
    assert M.round_bf16(np.array([-3.0 - 0.49 * 2 * u]))[0] == -3.0
    rng = np.random.default_rng(3)
    a = rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000)
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.round_bf16(a), ref)


def test_silu_and_derivative():
    z = np.linspace(-12, 12, 97)
    np.testing.assert_allclose(M.silu(z), z * expit(z), rtol=1e-14, atol=1e-300)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(M.dsilu(z), fd, rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("with_lin", [False, True])
def test_gradient_central_differences(with_lin):
    rng = np.random.default_rng(11)
    p = random_params(5)
    head = dict(HEAD)
    if with_lin:
        head["lin"] = 0.01 * rng.standard_normal((4, 6))
    x, qt = _inputs(7, 12)
    loss, g = M.loss_grad(p, x, qt, head)
    # indices in every parameter block (weights and biases of all 5 layers)
    offs = np.cumsum([0] + [r * c + r for r, c in M.LAYERS])
    idx = []
    for l, (r, c) in enumerate(M.LAYERS):
        idx += list(offs[l] + rng.integers(0, r * c, 8))
        idx += list(offs[l] + r * c + rng.integers(0, r, 4))
    # fourth-order central differences: truncation O(h^4), rounding ~ eps L / h
    h = 1e-4

    def f(i, d):
        pd = p.copy()
        pd[i] += d
        return M.loss_grad(pd, x, qt, head)[0]

    for i in idx:
        fd = (8 * (f(i, h) - f(i, -h)) - (f(i, 2 * h) - f(i, -2 * h))) / (12 * h)
        assert abs(g[i] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (i, g[i], fd)
    # the loss the gradient belongs to is the one defined: mean |q - qt|^2
    q, _ = M.forward(p, x, head)
    assert loss == pytest.approx(np.mean(np.sum((q - qt) ** 2, axis=1)), rel=1e-14)
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-15)


def test_zero_network_is_the_head():
    p = np.zeros(M.param_count())
    x, qt = _inputs(9, 4)
    lin = np.random.default_rng(2).standard_normal((4, 6)) * 1e-2
    head = dict(HEAD, lin=lin)
    q, _ = M.forward(p, x, head)
    xs = x * HEAD["in_scale"]
    u = HEAD["q0"] + xs @ lin.T
    np.testing.assert_allclose(q, u / np.linalg.norm(u, axis=1, keepdims=True), atol=1e-15)
    # with zero weights only the output bias has a gradient
    _, g = M.loss_grad(p, x, qt, head)
    assert np.all(g[:-4] == 0.0) and np.any(g[-4:] != 0.0)


def test_rotate_matches_rodrigues():
    rng = np.random.default_rng(8)
    for _ in range(20):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        th = rng.uniform(-math.pi, math.pi)
        v = rng.standard_normal(3)
        q = np.array([[math.cos(th / 2), *(n * math.sin(th / 2))]])
        rod = v * math.cos(th) + np.cross(n, v) * math.sin(th) + n * np.dot(n, v) * (1 - math.cos(th))
        np.testing.assert_allclose(M.rotate(q, v[:, None])[:, 0], rod, atol=1e-14)


def test_quat_from_images_all_branches():
    rng = np.random.default_rng(9)
    qs = [rng.standard_normal(4) for _ in range(40)]
    # rotations by ~pi about each axis exercise the branches with trace <= 0
    for ax in range(3):
        e = np.zeros(4)
        e[0] = 1e-3
        e[1 + ax] = 1.0
        qs.append(e)
        qs.append(-e)
    q = np.array(qs)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    ex = M.rotate(q, np.tile(np.array([[1.0], [0.0], [0.0]]), (1, len(q))))
    ey = M.rotate(q, np.tile(np.array([[0.0], [1.0], [0.0]]), (1, len(q))))
    r = M.quat_from_images(ex, ey)
    sgn = np.sign(np.sum(r * q, axis=1))[:, None]
    np.testing.assert_allclose(r * sgn, q, atol=1e-13)


def test_adam_first_step_closed_form():
    # first step: m^ = g, v^ = g^2, so every coordinate moves by lr g / (|g| + eps)
    rng = np.random.default_rng(1)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    p1, m, v = M.adam_step(p, np.zeros(50), np.zeros(50), g, 1, lr=1e-3, eps=1e-8)
    np.testing.assert_allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # a constant gradient keeps m^ = g, v^ = g^2 at every step
    for t in range(2, 6):
        p2, m, v = M.adam_step(p1, m, v, g, t, lr=1e-3, eps=0.0)
        np.testing.assert_allclose(p2 - p1, -1e-3 * np.sign(g), atol=1e-14)
        p1 = p2


def test_residual_gradient_central_differences():
    rng = np.random.default_rng(21)
    p = random_params(6)
    x, _ = _inputs(6, 22)
    r = rng.standard_normal((6, 4))
    loss, g = M.residual_loss_grad(p, x, r, HEAD["in_scale"])
    offs = np.cumsum([0] + [a * b + a for a, b in M.LAYERS])
    h = 1e-4

    def f(i, d):
        pd = p.copy()
        pd[i] += d
        return M.residual_loss_grad(pd, x, r, HEAD["in_scale"])[0]

    for l, (a, b) in enumerate(M.LAYERS):
        for i in list(offs[l] + rng.integers(0, a * b, 6)) + list(offs[l] + a * b + rng.integers(0, a, 3)):
            fd = (8 * (f(i, h) - f(i, -h)) - (f(i, 2 * h) - f(i, -2 * h))) / (12 * h)
            assert abs(g[i] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (i, g[i], fd)
    y, _ = M.network(p, x * HEAD["in_scale"])
    assert loss == pytest.approx(np.mean(np.sum((y - r) ** 2, axis=1)), rel=1e-14)


def test_bf16_gradient_storage_rounds_each_stage_once():
    """bf16_grads stores dL/dy, every SiLU'(z) and every dL/dz in bfloat16
    and changes nothing else: the output layer's gradient is exactly the one
    computed from the rounded dL/dy, the last hidden layer's exactly the one
    from the rounded dL/dz = bf16(dL/da * bf16(SiLU'(z))), every block moves by
    about the bf16 resolution (not more: relative L2 change below 2^-6, not
    zero), and a dL/dy already in bf16 reproduces the stored values."""
    rng = np.random.default_rng(41)
    p = random_params(9)
    x, _ = _inputs(64, 42)
    r = rng.standard_normal((64, 4))
    y, c = M.network(p, x * HEAD["in_scale"], bf16=True)
    gy = 2.0 * (y - r) / 64
    g0 = M.backward(c, gy)
    g1 = M.backward(c, gy, bf16_grads=True)
    offs = np.cumsum([0] + [a * b + a for a, b in M.LAYERS])
    gyr = M.round_bf16(gy)
    assert np.array_equal(g1[offs[4]:offs[5]], np.concatenate([(gyr.T @ c["acts"][4]).ravel(), gyr.sum(axis=0)]))
    W5, _ = c["layers"][4]
    z3 = c["zs"][3]
    s3 = 1.0 / (1.0 + np.exp(-z3))
    gz3 = M.round_bf16((gyr @ c["rd"](W5)) * M.round_bf16(s3 * (1.0 + z3 * (1.0 - s3))))
    assert np.array_equal(g1[offs[3]:offs[4]], np.concatenate([(gz3.T @ c["acts"][3]).ravel(), gz3.sum(axis=0)]))
    for l in range(5):
        a, b = offs[l], offs[l + 1]
        rel = np.linalg.norm(g1[a:b] - g0[a:b]) / np.linalg.norm(g0[a:b])
        assert 0.0 < rel < 2.0 ** -6, (l, rel)
    assert np.array_equal(M.backward(c, gyr, bf16_grads=True), g1)
    _, g2 = M.residual_loss_grad(p, x, r, HEAD["in_scale"], bf16=True, bf16_grads=True)
    _, g3 = M.residual_loss_grad(p, x, r, HEAD["in_scale"], bf16=True)
    assert not np.array_equal(g2, g3)


def test_split_bf16_resolution():
    """hi = bf16(v) exactly, and hi + lo resolves v to 2^-17 relative
    (two 8-bit significands)."""
    rng = np.random.default_rng(5)
    v = (rng.standard_normal(50000) * 10.0 ** rng.integers(-3, 3, 50000)).astype(np.float32)
    s = M.split_bf16(v)
    vv = v.astype(np.float64)
    assert np.all(np.abs(s - vv) <= 2.0 ** -17 * np.abs(vv))
    hi = M.round_bf16(v)
    assert np.all(np.abs(s - hi) <= 2.0 ** -8 * np.abs(vv))
    assert np.abs(s - vv).max() > 0                  # not the identity


def test_polynomial_head_terms():
    rng = np.random.default_rng(2)
    xs = rng.standard_normal((5, 6))
    terms = [(), (0,), (1, 2), (3, 3, 5)]
    coef = rng.standard_normal((4, 4))
    ref = (coef[:, 0][None, :] + np.outer(xs[:, 0], coef[:, 1]) + np.outer(xs[:, 1] * xs[:, 2], coef[:, 2])
           + np.outer(xs[:, 3] ** 2 * xs[:, 5], coef[:, 3]))
    np.testing.assert_allclose(M.poly(terms, coef, xs), ref, rtol=1e-14, atol=1e-14)
