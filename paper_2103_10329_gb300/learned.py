"""Training and use of the learned preconditioner correction.

Pairs come from the method itself: on random phantoms the multigrid
iteration runs as usual, and at grid 0 of each iteration the step alpha d of
the preconditioned Landweber step (input) and the error e = truth - mu of the
estimate it would update (target) are recorded, both divided by the RMS of
alpha d (the scale the network sees at inference).  The network is trained
on random crops by its own forward/backward kernels and Adam; the data
handling here (crops, batching) is host orchestration over device tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mgct, synth


def make_case(n: int, nu: int, views: int, levels: int, seed: int, count: int = 20,
              axis=(0.04, 0.2), device="cuda"):
    """A random ellipsoid phantom, its geometry and its projection data."""
    th, z = synth.trajectory(views, seed + 1)
    pitch = synth.default_pitch(nu)
    ph = synth.ellipsoids(count, seed, axis_lo=axis[0], axis_hi=axis[1])
    truth = synth.voxelize_ellipsoids(ph, n, supersample=2, device=device, dtype=torch.float32)
    geom = mgct.Geometry(n, nu, nu, th, z, pitch, levels=levels)
    b = mgct.project(geom, truth)
    return geom, b, truth


def generate_pairs(cases, iters: int = 2, storage=torch.float32):
    """[(x, t)] per case and iteration, float32 [n][n][n] device tensors."""
    pairs = []
    for geom, b, truth in cases:
        rec = mgct.Reconstructor(geom)
        rec.prepare(b)
        ws = mgct.workspace(geom, mgct.WS_LANDWEBER, 0)
        vol = torch.zeros_like(truth)
        step = torch.empty_like(truth)
        for _ in range(iters):
            if geom.levels > 1:
                mgct.multigrid_coarse(geom, vol, rec.ws, storage=storage)
            mgct.landweber_direction(geom, vol, b, ws=ws, out=step, storage=storage)
            s = float(torch.sqrt(torch.mean(step.double() ** 2)))
            if s > 0:
                pairs.append(((step / s).contiguous(), ((truth - vol) / s).contiguous()))
            mgct.axpy(1.0, step, vol)
    return pairs


def train(net: mgct.Net, pairs, steps: int = 300, crop: int = 32, batch: int = 4, lr: float = 1e-3,
          seed: int = 0, log_every: int = 0, decay_at: float = 0.7, decay: float = 0.3):
    """Adam on random crops, the learning rate multiplied by `decay` after
    the fraction `decay_at` of the steps; returns the loss history (host
    floats, one per log interval)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = pairs[0][0].shape[0]
    c = min(crop, n)
    x = torch.empty((batch, c, c, c), device="cuda")
    t = torch.empty_like(x)
    hist = []
    for it in range(steps):
        for j in range(batch):
            k = int(torch.randint(len(pairs), (1,), generator=g))
            o = torch.randint(n - c + 1, (3,), generator=g).tolist()
            px, pt = pairs[k]
            x[j] = px[o[0]:o[0] + c, o[1]:o[1] + c, o[2]:o[2] + c]
            t[j] = pt[o[0]:o[0] + c, o[1]:o[1] + c, o[2]:o[2] + c]
        loss = net.forward_backward(x, t)
        net.adam_step(lr if it < decay_at * steps else lr * decay)
        if log_every and (it % log_every == 0 or it == steps - 1):
            hist.append(float(loss.item()))
    return hist


def reconstruct(geom, b, iters: int = 2, net: mgct.Net | None = None, storage=torch.float32):
    """`iters` multigrid iterations from zero, with the learned step on grid 0
    when a network is given."""
    rec = mgct.Reconstructor(geom)
    rec.prepare(b)
    vol = torch.zeros((geom.n,) * 3, device="cuda")
    for _ in range(iters):
        if net is None:
            rec.iterate(vol, storage=storage)
        else:
            rec.iterate_learned(vol, net, storage=storage)
    return vol
