"""A preconditioner derived from the measured point-spread function of A^T A.

Eq. 5 is a fixed 3x3x3 approximate deconvolution; Sec. 3 of the paper notes
that it has zero response to a constant and asks for more rigorously derived
kernels.  Here the point-spread function h = A^T A e_j of the actual
geometry is measured at a few voxels j with the library's own operators,
averaged, and a 3x3x3 kernel k is fitted by least squares so that the
correlation k * h is as close as possible to a unit impulse over the window
of h.  The kernel is constrained to the symmetries of a circular trajectory
(x <-> y, x -> -x, y -> -y, z -> -z): six coefficients, by the distance class
of the offset (centre, x/y face, z face, in-plane edge, out-of-plane edge,
corner).  The measurement runs on the GPU; the fit is a host least-squares
problem of six unknowns, done once per geometry.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mgct


def measure_psf(geom: "mgct.Geometry", points, half: int = 5) -> np.ndarray:
    """Mean of (A^T A e_j) over the voxels `points` (j = (z, y, x) indices),
    each cut to the (2 half + 1)^3 window around j and scaled to a unit
    centre value.  float64 [2 half + 1]^3."""
    n = geom.n
    acc = np.zeros((2 * half + 1,) * 3)
    e = torch.zeros((n, n, n), device="cuda")
    for (z, y, x) in points:
        if not all(half <= c < n - half for c in (z, y, x)):
            raise ValueError("PSF points must lie at least `half` voxels inside the volume")
        e.zero_()
        e[z, y, x] = 1.0
        h = mgct.backproject(geom, mgct.project(geom, e))
        w = h[z - half:z + half + 1, y - half:y + half + 1, x - half:x + half + 1].double().cpu().numpy()
        acc += w / w[half, half, half]
    return acc / len(points)


def _classes() -> np.ndarray:
    """Class index (0..5) of each offset of a 3x3x3 kernel [dz][dy][dx]."""
    c = np.zeros((3, 3, 3), dtype=int)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nxy = abs(dx) + abs(dy)
                if dz == 0:
                    k = (0, 1, 3)[nxy]            # centre, x/y face, in-plane edge
                else:
                    k = (2, 4, 5)[nxy]            # z face, out-of-plane edge, corner
                c[dz + 1, dy + 1, dx + 1] = k
    return c


def fit_kernel(h: np.ndarray) -> np.ndarray:
    """Least-squares symmetric 3x3x3 kernel k with (k correlated with h) ~ delta
    over the window of h (zero outside it), scaled to a unit centre
    coefficient (the line search fixes the step's scale).  float64 [3][3][3]."""
    h = np.asarray(h, dtype=np.float64)
    m = h.shape[0]
    half = m // 2
    cls = _classes()
    pad = np.zeros((m + 2,) * 3)
    pad[1:-1, 1:-1, 1:-1] = h
    # column c: sum over the offsets d of class c of h(p + d), p over the window
    cols = np.zeros((m ** 3, 6))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                cols[:, cls[dz, dy, dx]] += pad[dz:dz + m, dy:dy + m, dx:dx + m].reshape(-1)
    target = np.zeros((m,) * 3)
    target[half, half, half] = 1.0
    coef, *_ = np.linalg.lstsq(cols, target.reshape(-1), rcond=None)
    k = coef[cls]
    return k / k[1, 1, 1]


def derived_preconditioner(geom: "mgct.Geometry", half: int = 5, offsets=(0.0, 0.2, -0.2)) -> tuple:
    """Measure the PSF at the centre and at voxels displaced by `offsets`
    (fractions of the side along x, y and z), fit the kernel; returns
    (kernel [3][3][3], mean PSF)."""
    n = geom.n
    c = n // 2
    pts = []
    for f in offsets:
        d = int(round(f * n))
        pts.append((c, c, c + d))
        if d:
            pts.append((c + d // 2, c + d, c))
    h = measure_psf(geom, pts, half)
    return fit_kernel(h), h
