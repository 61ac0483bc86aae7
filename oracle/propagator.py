"""CPU oracle of the learned density propagator (test infrastructure only).

The network maps the per-species density meshes at the last two true field
refreshes, x = ((phi_A, phi_B)(t - K), (phi_A, phi_B)(t)) -- 4 channels on the
periodic mesh -- to the change (phi_A, phi_B)(t + K) - (phi_A, phi_B)(t).  Its
input channels are features(x) = (s (phi(t) - phi(t - K)), phi(t)) per
species, s a fixed change scale:

    h1 = SiLU(conv(features(x), W1) + b1)      4 -> 16 channels
    h2 = SiLU(conv(h1, W2) + b2)    16 -> 16
    y  = (conv(h2, W3) + b3) / s    16 ->  2

conv is a 3x3x3 periodic convolution (cross-correlation, as in deep-learning
libraries): out[co](n) = sum_ci sum_d W[d][ci][co] in[ci](n + d), with the
27 offsets d = (dz, dy, dx) in {-1, 0, 1}^3 in z-major order.  Meshes are
[C][Mz][My][Mx].  FP64 throughout; the loss is s^2 times the mean squared
error of y over all voxels and output channels (the error of the last
layer's output against the scaled change).

Parity status: conv, SiLU and the whole network forward are pinned by closed
forms (delta kernels shift the input, periodic wrap, linearity, SiLU values);
every backward quantity is pinned against central finite differences of the
loss.  The learned network's predictions themselves are not pinned (they are
a fitted model); what they gain is measured against holding the last field.
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
LAYERS = [(4, 16, True), (16, 16, True), (16, 2, False)]


def shift(a, d):
    """a(n + d) on the periodic mesh, for a [..., Mz, My, Mx] array and d = (dz, dy, dx)."""
    dz, dy, dx = d
    return np.roll(a, shift=(-dz, -dy, -dx), axis=(-3, -2, -1))


def conv(x, W, b=None):
    """x [Ci][Mz][My][Mx], W [27][Ci][Co] -> [Co][Mz][My][Mx]."""
    out = np.zeros((W.shape[2],) + x.shape[1:])
    for k, d in enumerate(OFFSETS):
        xs = shift(x, d)
        out += np.einsum("imnl,io->omnl", xs, W[k])
    if b is not None:
        out += b[:, None, None, None]
    return out


def conv_backward(x, W, gy):
    """Gradients of sum(gy * conv(x, W)) with respect to x, W and the bias."""
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for k, d in enumerate(OFFSETS):
        xs = shift(x, d)
        gW[k] = np.einsum("imnl,omnl->io", xs, gy)
        # d/dx[i](m) of sum_n gy(n) x(n + d) = gy(m - d)
        gx += np.einsum("omnl,io->imnl", shift(gy, tuple(-c for c in d)), W[k])
    gb = gy.sum(axis=(1, 2, 3))
    return gx, gW, gb


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(seed=0):
    """He-style uniform initialisation (the GPU path receives these values)."""
    rng = np.random.default_rng(seed)
    params = []
    for ci, co, _ in LAYERS:
        lim = np.sqrt(6.0 / (27 * ci))
        params.append((rng.uniform(-lim, lim, size=(27, ci, co)), np.zeros(co)))
    params[-1] = (params[-1][0] * 0.1, params[-1][1])
    return params


def features(x, scale=1.0):
    """The network's input channels from x = (phi_A, phi_B at t - K, phi_A, phi_B
    at t): the scaled changes scale * (phi(t) - phi(t - K)) and the current
    phi(t), per species, formed in full precision before any rounding."""
    return np.stack([scale * (x[2] - x[0]), scale * (x[3] - x[1]), x[2], x[3]])


def forward(params, x, scale=1.0):
    """Returns the predicted change y and the per-layer (input, pre-activation) cache."""
    cache = []
    h = features(x, scale)
    for (W, b), (_, _, act) in zip(params, LAYERS):
        z = conv(h, W, b)
        cache.append((h, z))
        h = silu(z) if act else z
    return h / scale, cache


def loss(params, x, target, scale=1.0):
    y, _ = forward(params, x, scale)
    return float(np.mean((scale * y - scale * target) ** 2))


def backward(params, x, target, scale=1.0):
    """Loss and its gradients [(gW, gb) per layer] by back-propagation."""
    y, cache = forward(params, x, scale)
    L = float(np.mean((scale * y - scale * target) ** 2))
    g = 2.0 * (scale * y - scale * target) / y.size
    grads = [None] * len(params)
    for li in reversed(range(len(params))):
        h, z = cache[li]
        if LAYERS[li][2]:
            g = g * silu_grad(z)
        gx, gW, gb = conv_backward(h, params[li][0], g)
        grads[li] = (gW, gb)
        g = gx
    return L, grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2015) of every tensor, in place; state = (t, m, v)."""
    t, m, v = state
    t += 1
    new = []
    for li, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        out = []
        for j, (p, g) in enumerate(((W, gW), (b, gb))):
            m[li][j] = b1 * m[li][j] + (1 - b1) * g
            v[li][j] = b2 * v[li][j] + (1 - b2) * g * g
            mh = m[li][j] / (1 - b1 ** t)
            vh = v[li][j] / (1 - b2 ** t)
            out.append(p - lr * mh / (np.sqrt(vh) + eps))
        new.append(tuple(out))
    return new, (t, m, v)


def adam_state(params):
    return (0, [[np.zeros_like(W), np.zeros_like(b)] for W, b in params],
            [[np.zeros_like(W), np.zeros_like(b)] for W, b in params])


def smooth(phi, passes):
    """The periodic binomial filter (1/4, 1/2, 1/4) along x, y and z in turn,
    passes times, of a [..., Mz, My, Mx] mesh (the smoothed-density variant of
    the propagator study)."""
    out = np.asarray(phi, dtype=np.float64).copy()
    for _ in range(passes):
        for axis in (-1, -2, -3):
            out = 0.25 * (np.roll(out, 1, axis=axis) + np.roll(out, -1, axis=axis)) + 0.5 * out
    return out
