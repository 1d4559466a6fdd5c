"""FP64 NumPy reference of the learned one-turn spin map -- TEST
INFRASTRUCTURE ONLY (tests, smoke and the bench's reference leg).

Network: 6 -> 256 -> 256 -> 256 -> 256 -> 4, SiLU activations, head
q = normalise(q0 + P(x) + s y) with x the per-coordinate scaled input, P a
polynomial (a linear term L x, or monomials with coefficients) and y the
network output; losses mean_b |q_b - q_target_b|^2 (quaternion) and
mean_b |y_b - r_b|^2 (residual regression).  Flattened parameter order:
W1[256][6], b1, W2[256][256], b2, W3, b3, W4, b4, W5[4][256], b5.

`bf16=True` rounds the weights and every hidden activation to bfloat16 (round
to nearest even) and represents the scaled input as the two-term bf16 split of
its float32 value, keeping FP64 arithmetic: the storage precision of the GPU
kernels without their FP32 accumulation order.  `bf16_grads=True` also stores
the back-propagated dL/dy, every dL/dz and every SiLU derivative SiLU'(z) in
bfloat16, as the kernels do between their gradient GEMMs (the forward pass
keeps SiLU'(z) in bf16, the activations' storage precision, for the
backward pass; the arithmetic stays FP64).
"""
from __future__ import annotations

import numpy as np

LAYERS = [(256, 6), (256, 256), (256, 256), (256, 256), (4, 256)]


def param_count() -> int:
    return sum(r * c + r for r, c in LAYERS)


def unpack(p):
    out, o = [], 0
    for r, c in LAYERS:
        W = p[o:o + r * c].reshape(r, c)
        o += r * c
        b = p[o:o + r]
        o += r
        out.append((W, b))
    return out


def round_bf16(a):
    """Round float64 values to the nearest bfloat16 (ties to even)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def split_bf16(v):
    """Two-term bf16 representation of float32 values: hi = bf16(v),
    lo = bf16(v - hi); returns hi + lo (exact in float64)."""
    v = np.asarray(v, dtype=np.float32)
    hi = round_bf16(v).astype(np.float32)
    lo = round_bf16(v - hi)
    return hi.astype(np.float64) + lo


def scaled_input(x, in_scale, bf16):
    """The first layer's input.  With bf16 the kernels' representation: the
    float32 product x * in_scale split into bf16 hi + lo; else FP64 x * in_scale."""
    if bf16:
        return split_bf16(np.asarray(x, np.float32) * np.asarray(in_scale, np.float32))
    return np.asarray(x, dtype=np.float64) * np.asarray(in_scale, dtype=np.float64)


def network(p, a0, bf16=False):
    """The five layers from the scaled input a0 [B, 6]: y [B, 4] and the cache."""
    layers = unpack(np.asarray(p, dtype=np.float64))
    rd = round_bf16 if bf16 else (lambda a: a)
    a = a0
    acts, zs = [a], []
    for l in range(4):
        W, b = layers[l]
        z = a @ rd(W).T + b
        zs.append(z)
        a = rd(silu(z))
        acts.append(a)
    W5, b5 = layers[4]
    y = a @ rd(W5).T + b5
    return y, dict(layers=layers, acts=acts, zs=zs, rd=rd)


def backward(c, gy, bf16_grads=False):
    """Gradient (flattened, parameter order) from dL/dy [B, 4]; bf16_grads
    stores dL/dy, each SiLU'(z) and each dL/dz in bfloat16 before it is used."""
    rd = c["rd"]
    rg = round_bf16 if bf16_grads else (lambda a: a)
    grads = [None] * 5
    W5, _ = c["layers"][4]
    gy = rg(gy)
    grads[4] = (gy.T @ c["acts"][4], gy.sum(axis=0))
    ga = gy @ rd(W5)
    for l in range(3, -1, -1):
        gz = rg(ga * rg(dsilu(c["zs"][l])))
        W, _ = c["layers"][l]
        grads[l] = (gz.T @ c["acts"][l], gz.sum(axis=0))
        ga = gz @ rd(W)
    return np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])


def poly(terms, coef, xs):
    """P(x) [B, 4] = sum_f coef[:, f] prod_{i in terms[f]} x_i."""
    out = np.zeros((xs.shape[0], 4))
    for f, t in enumerate(terms):
        m = np.ones(xs.shape[0])
        for i in t:
            m = m * xs[:, i]
        out += m[:, None] * np.asarray(coef)[:, f][None, :]
    return out


def head_polynomial(head, xs):
    """P(x) of a head: 'lin' [4, 6] (linear term) or 'poly' = (terms, coef)."""
    if head.get("poly") is not None:
        terms, coef = head["poly"]
        return poly(terms, coef, xs)
    if head.get("lin") is not None:
        return xs @ np.asarray(head["lin"], dtype=np.float64).T
    return np.zeros((xs.shape[0], 4))


def forward(p, x, head, bf16=False):
    """q [B, 4] = normalise(q0 + P(x) + s y) and the cache.
    head: dict(q0[4], lin[4, 6] or poly=(terms, coef) or neither, scale, in_scale[6])."""
    y, c = network(p, scaled_input(x, head["in_scale"], bf16), bf16)
    xs = np.asarray(x, dtype=np.float64) * np.asarray(head["in_scale"], dtype=np.float64)
    u = np.asarray(head["q0"], dtype=np.float64)[None, :] + head_polynomial(head, xs) + head["scale"] * y
    nrm = np.linalg.norm(u, axis=1, keepdims=True)
    q = u / nrm
    c.update(u=u, nrm=nrm, q=q, y=y)
    return q, c


def loss_grad(p, x, qt, head, bf16=False, bf16_grads=False):
    """Loss mean_b |q_b - qt_b|^2 and its gradient (flattened, parameter order)."""
    q, c = forward(p, x, head, bf16)
    B = q.shape[0]
    d = q - qt
    loss = float((d * d).sum() / B)
    gq = 2.0 * d / B
    gu = (gq - q * (q * gq).sum(axis=1, keepdims=True)) / c["nrm"]
    return loss, backward(c, head["scale"] * gu, bf16_grads)


def residual_loss_grad(p, x, r, in_scale, bf16=False, bf16_grads=False):
    """Regression of the raw outputs: loss mean_b |y_b - r_b|^2 and its gradient."""
    y, c = network(p, scaled_input(x, in_scale, bf16), bf16)
    B = y.shape[0]
    d = y - r
    return float((d * d).sum() / B), backward(c, 2.0 * d / B, bf16_grads)


def quat_from_images(ex, ey):
    """Unit quaternions (scalar first) of rotations R given the images R x^,
    R y^ as [3, n] arrays (R z^ = R x^ x R y^)."""
    ez = np.cross(ex.T, ey.T).T
    R = np.stack([ex, ey, ez], axis=1)          # R[:, j, n] = column j
    R = np.transpose(R, (2, 0, 1))              # [n, 3, 3] with R[n][i][j]
    tr = np.trace(R, axis1=1, axis2=2)
    q = np.empty((R.shape[0], 4))
    for i in range(R.shape[0]):
        m = R[i]
        t = tr[i]
        if t > 0:
            s = 2.0 * np.sqrt(1.0 + t)
            q[i] = [0.25 * s, (m[2, 1] - m[1, 2]) / s, (m[0, 2] - m[2, 0]) / s, (m[1, 0] - m[0, 1]) / s]
        elif m[0, 0] > m[1, 1] and m[0, 0] > m[2, 2]:
            s = 2.0 * np.sqrt(1.0 + m[0, 0] - m[1, 1] - m[2, 2])
            q[i] = [(m[2, 1] - m[1, 2]) / s, 0.25 * s, (m[0, 1] + m[1, 0]) / s, (m[0, 2] + m[2, 0]) / s]
        elif m[1, 1] > m[2, 2]:
            s = 2.0 * np.sqrt(1.0 + m[1, 1] - m[0, 0] - m[2, 2])
            q[i] = [(m[0, 2] - m[2, 0]) / s, (m[0, 1] + m[1, 0]) / s, 0.25 * s, (m[1, 2] + m[2, 1]) / s]
        else:
            s = 2.0 * np.sqrt(1.0 + m[2, 2] - m[0, 0] - m[1, 1])
            q[i] = [(m[1, 0] - m[0, 1]) / s, (m[0, 2] + m[2, 0]) / s, (m[1, 2] + m[2, 1]) / s, 0.25 * s]
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def rotate(q, S):
    """Rotate vectors S [3, n] by unit quaternions q [n, 4] (S' = q S conj(q))."""
    w = q[:, 0]
    v = q[:, 1:].T
    t = 2.0 * np.cross(v.T, S.T).T
    return S + w * t + np.cross(v.T, t.T).T


def adam_step(p, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) at step t >= 1; returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
