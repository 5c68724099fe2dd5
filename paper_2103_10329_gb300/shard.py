"""View-sharded A and A^T across ranks, one process per GPU.

The views of a scan are independent (Eq. 1 sums along each ray of each
radiograph), so a rank that owns a contiguous range of views projects them
with no exchange, and A^T = sum over views splits into one partial volume
per rank, summed over the ranks.  The paper runs on an MPI framework over
several GPUs (Sec. 2, its ref. [12]) without describing it; this is the
partitioning of that sum for this library.

The partial volumes are summed in rank order by default (each rank gathers
every partial and adds them in order with the library's axpy kernel), so the
result is the same bit for bit on every rank and for every collective
algorithm; `ordered=False` hands the sum to the collective itself
(all_reduce, NCCL on GPUs).  Tensors on a CUDA device go through host memory
when the process group's backend is gloo.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import mgct


def view_range(n_views: int, rank: int, world: int) -> tuple[int, int]:
    """(first view, count) of rank `rank`'s contiguous share of n_views:
    the first n_views % world ranks take one view more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, extra = divmod(n_views, world)
    v0 = rank * base + min(rank, extra)
    return v0, base + (1 if rank < extra else 0)


def project_shard(geom, vol: torch.Tensor, rank: int, world: int, level: int = 0, **kw) -> torch.Tensor:
    """A vol over this rank's views (mgct.project); no exchange."""
    v0, cnt = view_range(geom.n_views, rank, world)
    return mgct.project(geom, vol, level=level, views=(v0, cnt, 1), **kw)


def _gather(t: torch.Tensor, world: int, group) -> list[torch.Tensor]:
    staged = t.device.type == "cuda" and dist.get_backend(group) == "gloo"
    src = t.cpu() if staged else t
    parts = [torch.empty_like(src) for _ in range(world)]
    dist.all_gather(parts, src, group=group)
    return [p.to(t.device) for p in parts] if staged else parts


def _add(x: torch.Tensor, y: torch.Tensor) -> None:
    """y += x (the library's axpy on the GPU)."""
    if y.device.type == "cuda":
        mgct.axpy(1.0, x, y)
    else:
        y.add_(x)


def backproject_sharded(geom, sino_local: torch.Tensor, rank: int, world: int, level: int = 0,
                        group=None, ordered: bool = True, backproject=None) -> torch.Tensor:
    """A^T over every view, each rank holding the sinogram of its own views
    (view_range): this rank's partial volume, then the sum over ranks.
    Returns the whole volume on every rank.  `backproject(geom, sino, level,
    views)` is the per-rank operator (mgct.backproject by default)."""
    v0, cnt = view_range(geom.n_views, rank, world)
    bp = backproject or (lambda g, y, lv, views: mgct.backproject(g, y, level=lv, views=views))
    partial = bp(geom, sino_local, level, (v0, cnt, 1))
    if world == 1:
        return partial
    if not ordered:
        staged = partial.device.type == "cuda" and dist.get_backend(group) == "gloo"
        buf = partial.cpu() if staged else partial
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
        return buf.to(partial.device) if staged else buf
    parts = _gather(partial, world, group)
    out = parts[0].clone()
    for p in parts[1:]:
        _add(p, out)
    return out
