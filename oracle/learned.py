"""FP64 oracle of the learned preconditioner correction network.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The network: four
3x3x3 convolutions at full resolution with zero padding, 1 -> 16 -> 32 -> 64
-> 1 channels, ReLU after the first three; prediction x + f(x) for the
scaled step x, loss mean((x + f(x) - t)^2).  Plain numpy: one einsum per
tap, the backward pass written out by hand.

`bf16=True` rounds, to bfloat16 (round to nearest even), exactly the tensors
the GPU stores in bfloat16: the network input, the weights, every hidden
activation and every back-propagated gradient; everything else is float64.
"""
from __future__ import annotations

import numpy as np

CIN = (1, 16, 32, 64)
COUT = (16, 32, 64, 1)
TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def param_count() -> int:
    return sum(27 * co * ci + co for ci, co in zip(CIN, COUT))


def unpack(p):
    """Flat float array -> list of (W [27, cout, cin], b [cout])."""
    p = np.asarray(p, dtype=np.float64)
    out, off = [], 0
    for ci, co in zip(CIN, COUT):
        w = p[off:off + 27 * co * ci].reshape(27, co, ci)
        off += 27 * co * ci
        b = p[off:off + co]
        off += co
        out.append((w, b))
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def bf16(x):
    """Round to bfloat16 (nearest even), returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _shift(x, dz, dy, dx):
    """y[.., z, y, x, :] = x[.., z+dz, y+dy, x+dx, :] with zero outside."""
    B, D, H, W, C = x.shape
    p = np.zeros((B, D + 2, H + 2, W + 2, C))
    p[:, 1:-1, 1:-1, 1:-1] = x
    return p[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]


def conv(x, w, b=None):
    """out[p, co] = sum_tap sum_ci x[p + tap, ci] w[tap, co, ci] + b[co]; x [B, D, H, W, C]."""
    out = np.zeros(x.shape[:-1] + (w.shape[1],))
    for k, (dz, dy, dx) in enumerate(TAPS):
        out += np.einsum("bzyxc,oc->bzyxo", _shift(x, dz, dy, dx), w[k])
    return out + (b if b is not None else 0.0)


def conv_data_grad(g, w):
    """d/dx of sum(g * conv(x, w)): gin[p, ci] = sum_tap g[p - tap] w[tap, :, ci]."""
    out = np.zeros(g.shape[:-1] + (w.shape[2],))
    for k, (dz, dy, dx) in enumerate(TAPS):
        out += np.einsum("bzyxo,oc->bzyxc", _shift(g, -dz, -dy, -dx), w[k])
    return out


def conv_weight_grad(x, g):
    """d/dw of sum(g * conv(x, w)): dw[tap, co, ci] = sum_p g[p, co] x[p + tap, ci]."""
    return np.stack([np.einsum("bzyxo,bzyxc->oc", g, _shift(x, dz, dy, dx)) for dz, dy, dx in TAPS])


def forward(params, x, bf=False):
    """x: [B, D, H, W] scaled step.  Returns (y [B, D, H, W], cache)."""
    r = bf16 if bf else (lambda a: a)
    layers = [(r(w), b) for w, b in unpack(params)]
    a = r(x[..., None])
    acts = [a]
    for l, (w, b) in enumerate(layers):
        z = conv(a, w, b)
        if l < 3:
            a = r(np.maximum(z, 0.0))
            acts.append(a)
        else:
            y = z[..., 0]
    return y, (layers, acts)


def loss_and_grads(params, x, t, bf=False):
    """Loss mean((x + f(x) - t)^2) and its gradient w.r.t. the flat params."""
    r = bf16 if bf else (lambda a: a)
    y, (layers, acts) = forward(params, x, bf)
    res = x + y - t
    n = res.size
    loss = float(np.mean(res * res))
    g = r((2.0 / n) * res)[..., None]          # dL/d(output of layer 3)
    grads = [None] * 4
    for l in range(3, -1, -1):
        w, _ = layers[l]
        grads[l] = (conv_weight_grad(acts[l], g), g.sum(axis=(0, 1, 2, 3)))
        if l > 0:
            g = r(conv_data_grad(g, w) * (acts[l] > 0))
    return loss, pack(grads)
