"""torch.autograd wrappers of the projector and back-projector (Sec. 1:
geometry drift estimated jointly with the image).  Forward and backward run
in libmgct's kernels: the backward of A is A^T for the volume and the
geometry-gradient kernel for the per-view drift parameters; the backward of
A^T is A."""
from __future__ import annotations

import torch

from . import mgct


def _sync_drift(geom: mgct.Geometry, phi: torch.Tensor | None):
    if phi is not None:
        geom.set_drift(phi.detach().to("cpu", torch.float64).numpy())


class Project(torch.autograd.Function):
    """y = A(phi) vol for all views of grid `level`; phi: [K, 5] drift
    (ds_u, ds_v, dd_u, dd_v in fine pixels, psi in radians) or None."""

    @staticmethod
    def forward(ctx, vol, phi, geom, level):
        _sync_drift(geom, phi)
        ctx.geom, ctx.level = geom, level
        ctx.save_for_backward(vol, phi if phi is not None else torch.empty(0))
        ctx.has_phi = phi is not None
        return mgct.project(geom, vol.contiguous(), level=level)

    @staticmethod
    def backward(ctx, gout):
        vol, phi = ctx.saved_tensors
        geom, level = ctx.geom, ctx.level
        _sync_drift(geom, phi if ctx.has_phi else None)
        gout = gout.contiguous().to(torch.float32)
        gvol = mgct.backproject(geom, gout, level=level) if ctx.needs_input_grad[0] else None
        gphi = None
        if ctx.has_phi and ctx.needs_input_grad[1]:
            gphi = mgct.geometry_grad(geom, vol.contiguous(), gout, level=level).to(phi.dtype).to(phi.device)
        return gvol, gphi, None, None


class Backproject(torch.autograd.Function):
    """vol = A^T y (fixed geometry); its backward is A."""

    @staticmethod
    def forward(ctx, y, geom, level):
        ctx.geom, ctx.level = geom, level
        return mgct.backproject(geom, y.contiguous(), level=level)

    @staticmethod
    def backward(ctx, gvol):
        return mgct.project(ctx.geom, gvol.contiguous().to(torch.float32), level=ctx.level), None, None


def project(vol, geom, phi=None, level: int = 0):
    return Project.apply(vol, phi, geom, level)


def backproject(y, geom, level: int = 0):
    return Backproject.apply(y, geom, level)
