"""The propagator oracle evaluated on the values the GPU kernels consume.

The GPU network rounds to BF16 at fixed points: the input features (formed
in FP32), every weight, the two hidden activations after SiLU, the loss
gradient d / V and the back-propagated gradients after the SiLU derivative.
Applying the same roundings here, between calls to the unchanged FP64 oracle
primitives (oracle/propagator.py: conv, conv_backward, silu, silu_grad),
leaves as the only differences from the GPU its FP32 accumulation order and
the rare hidden value whose FP32 pre-activation rounds to the neighbouring
BF16 number.  Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from oracle import propagator as P


def bf16(a):
    """Round to BF16 (nearest, ties to even) from FP32, returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def rounded_params(params):
    """BF16 weights and FP32 biases, as the kernels hold them."""
    return [(bf16(W), np.asarray(b, np.float32).astype(np.float64)) for W, b in params]


def features32(x, scale):
    """The input channels formed in FP32 (as the GPU forms them) and rounded to BF16."""
    x = np.asarray(x, np.float32)
    s = np.float32(scale)
    return bf16(np.stack([s * (x[2] - x[0]), s * (x[3] - x[1]), x[2], x[3]]))


def forward(params, x, scale=1.0):
    """y (the predicted change) and the per-layer inputs and pre-activations."""
    Wr = rounded_params(params)
    h = features32(x, scale)
    hs, zs = [], []
    for (W, b), (_, _, act) in zip(Wr, P.LAYERS):
        z = P.conv(h, W, b)
        hs.append(h)
        zs.append(z)
        h = bf16(P.silu(z)) if act else z
    return h / scale, hs, zs, Wr


def backward(params, x, phi_next, scale=1.0):
    """Loss and [(gW, gb) per layer] with the GPU's rounding points."""
    y, hs, zs, Wr = forward(params, x, scale)
    V = y[0].size
    x32 = np.asarray(x, np.float32)
    d = np.asarray(y * scale, np.float32) - np.float32(scale) * (
        np.asarray(phi_next, np.float32) - x32[2:])
    d64 = d.astype(np.float64)
    loss = float(np.sum(d64 * d64) / (2.0 * V))
    g = bf16(d / np.float32(V))
    grads = [None] * len(Wr)
    for li in reversed(range(len(Wr))):
        gx, gW, gb = P.conv_backward(hs[li], Wr[li][0], g)
        grads[li] = (gW, gb)
        if li == 0:
            break
        g = bf16(gx * P.silu_grad(zs[li - 1]))
    return loss, grads
