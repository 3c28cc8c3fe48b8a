"""FP64 reference of the surrogate network (test infrastructure only).

MLP n_in -> W -> W -> W -> n_out, SiLU activations, parameters laid out as
[W1 b1 W2 b2 W3 b3 W4 b4] with W_l [out_pad][in_pad] row-major, inputs and outputs padded
to multiples of 16.  Loss: mean over the batch of (o_0 - y_0)^2 + mean_{j>=1} (o_j - y_j)^2.
Forward and backward are written out by hand (chain rule, SiLU'(z) = s(1 + z(1 - s)),
s = sigmoid(z)).  With ``bf16=True`` the inputs, weights, activations and backpropagated
pre-activation gradients are rounded to bfloat16 where the GPU stores them in bfloat16, so
the remaining difference to the GPU is FP32 accumulation order.
"""
from __future__ import annotations

import numpy as np


def pad16(n: int) -> int:
    return (n + 15) // 16 * 16


def to_bf16(a) -> np.ndarray:
    """Round float64/float32 values to the nearest bfloat16 (ties to even), returned as FP64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    u = ((u + rounding) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def layout(n_in: int, n_out: int, width: int):
    ins = [pad16(n_in), width, width, width]
    outs = [width, width, width, pad16(n_out)]
    off, lay = 0, []
    for i, o in zip(ins, outs):
        lay.append((off, o, i, off + o * i))
        off += o * i + o
    return lay, off


def unpack(params, n_in, n_out, width):
    lay, total = layout(n_in, n_out, width)
    params = np.asarray(params, dtype=np.float64)
    assert params.size == total
    return [(params[w:w + o * i].reshape(o, i), params[b:b + o]) for (w, o, i, b) in lay]


def silu(z):
    return z / (1.0 + np.exp(-z))


def forward(params, x, n_in, n_out, width, bf16=False, scaling=None):
    """Returns (outputs [B, n_out], cache for backward).  scaling = (in_shift, in_mul,
    out_shift, out_mul): the network sees (x - in_shift) in_mul and reports o out_mul +
    out_shift (default: identity)."""
    layers = unpack(params, n_in, n_out, width)
    B = x.shape[0]
    X = np.zeros((B, pad16(n_in)))
    if scaling is not None:
        X[:, :n_in] = (np.asarray(x[:, :n_in], dtype=np.float64) - scaling[0]) * scaling[1]
    else:
        X[:, :n_in] = x[:, :n_in]
    rnd = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    h = rnd(X)
    hs, zs = [h], []
    for l, (W, b) in enumerate(layers):
        z = h @ rnd(W).T + b
        zs.append(z)
        if l < 3:
            h = rnd(silu(z))
            hs.append(h)
    o = zs[-1][:, :n_out]
    if scaling is not None:
        o = o * scaling[3] + scaling[2]
    return o, (layers, hs, zs, rnd)


def loss_and_grads(params, x, y, n_in, n_out, width, bf16=False, scaling=None):
    """Loss and the gradient of every parameter (flat array in the parameter layout); with
    scaling the loss compares the raw network outputs with standardised targets
    (y - out_shift) / out_mul."""
    _, (layers, hs, zs, rnd) = forward(params, x, n_in, n_out, width, bf16, scaling)
    out = zs[-1][:, :n_out]
    B = x.shape[0]
    wts = np.full(n_out, 1.0 / (n_out - 1)); wts[0] = 1.0
    yt = np.asarray(y[:, :n_out], dtype=np.float64)
    if scaling is not None:
        yt = (yt - scaling[2]) / scaling[3]
    d = out - yt
    loss = float(np.sum(wts * d * d) / B)
    dO = np.zeros_like(zs[-1])
    dO[:, :n_out] = 2.0 * wts * d / B
    dz = rnd(dO)
    grads = []
    for l in range(3, -1, -1):
        W, b = layers[l]
        grads.append((dz.T @ hs[l], dz.sum(0)))
        if l == 0:
            break
        dh = dz @ rnd(W)
        z = zs[l - 1]
        s = 1.0 / (1.0 + np.exp(-z))
        dz = rnd(dh * s * (1.0 + z * (1.0 - s)))
    grads = grads[::-1]
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, flat
