#!/usr/bin/env python
"""Benchmark of the preconditioned multigrid Landweber reconstruction on one
GB300 (replicas only across GPUs).

One step = one multigrid iteration of Alg. 1 at grid 0 (restrict, recurse,
OS-EMTR on the coarsest grid, prolongate, and on every other grid one
preconditioned Landweber step: A with residual, A^T, the Eq. 5 filter, a
second A for the line search, the update).

Headline workload (the largest configuration): a 1024^3 volume of 100 random
ellipsoids plus a porous texture, 1536x1536 detector, 2880 views on the
space-filling trajectory, 4 grids, Poisson noise at 1e4 photons per ray.
The 256^3 / 384^2 / 720-view workload (data projected from a 2x finer
phantom) follows as a secondary line with the time-to-accuracy runs.

The value is whole-job A+A^T throughput in GUPS: voxel-view updates (n_g^3 x
views for every A and A^T call of the step, on every grid) per second.
`--impl reference` times the FP64 CPU oracle (A and A^T on a sample of views
and rows) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "A+A^T GUPS & % BW roofline; sec to RMSE≤1e-3 (learned/BF16 vs plain FP32)"
WORKLOADS = {
    # name: n, nu, views, levels, ellipsoids, axis range, texture, photons;
    # fine: the data are projected from a phantom `fine` times finer (1: the
    # reconstruction grid itself)
    "c5": dict(n=1024, nu=1536, views=2880, levels=4, count=100, axis=(0.01, 0.08), texture=True,
               photons=1e4, fine=1),
    "c3": dict(n=512, nu=768, views=1440, levels=3, count=50, axis=(0.04, 0.2), texture=False, photons=0,
               fine=2),
    "c2": dict(n=256, nu=384, views=720, levels=3, count=200, axis=(0.01, 0.08), texture=True,
               photons=1e4, fine=2),
    "c1": dict(n=64, nu=96, views=90, levels=2, count=10, axis=(0.04, 0.2), texture=False, photons=0, fine=2),
    # half the views of c2, noise- and texture-free: the small case for ncu captures
    "c2h": dict(n=256, nu=384, views=360, levels=3, count=50, axis=(0.01, 0.08), texture=False, photons=0,
                fine=2),
}
SEED = 2103
FP32_LANES_PER_SM, SMS = 128, 152


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(name):
    w = WORKLOADS[name]
    return {"workload": f"{w['n']}^3 volume, {w['count']} ellipsoids" + (" + porous texture" if w["texture"] else "")
            + f", {w['nu']}x{w['nu']} detector, {w['views']} space-filling views, {w['levels']} grids"
            + (f", Poisson {w['photons']:.0e} photons/ray" if w["photons"] else ", noise-free")
            + (", data projected from a 2x finer phantom" if w["fine"] == 2 else
               ", data projected from the phantom on the reconstruction grid"),
            "n": w["n"], "detector": [w["nu"], w["nu"]], "views": w["views"], "levels": w["levels"],
            "iteration": "Alg. 1 multigrid, Landweber with line search, OS-EMTR M=8 on the coarsest grid",
            "l2": "inputs larger than L2 (sinogram %d MB)" % (w["views"] * w["nu"] ** 2 * 4 // 2 ** 20)}


def aggregate(ms_local: float, units_local: float, device="cpu"):
    """Whole-job timing over replicas: (max of ms over ranks, sum of units),
    through torch.distributed when it is initialised (NCCL on the GPU machine,
    gloo in the CPU tests), else the local values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms_local, units_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def units_per_step(n, views, levels):
    """Voxel-view updates of the A / A^T calls of one multigrid iteration."""
    u = 0
    for g in range(levels):
        ng = n >> g
        if levels == 1 or g < levels - 1:
            u += 3 * ng ** 3 * views   # A (residual), A^T, A (line search)
        else:
            u += 2 * ng ** 3 * views   # OS-EMTR: A and two-channel A^T over all subsets
    return u


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        load = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work of A / A^T: nonzeros of the matrix (4 bilinear taps per
# in-volume sample), counted per ray from the plane range where the ray's
# crossing lies inside (-1, n) on both in-plane axes
# ---------------------------------------------------------------------------
def count_nnz(theta, z, pitch, n, nu, nv, src_axis=2.0, src_det=4.0, device="cuda"):
    import torch
    h = 1.0 / n
    ic = 0.5 * (n - 1)
    total = 0.0
    ju = torch.arange(nu, device=device, dtype=torch.float64) - 0.5 * (nu - 1)
    jv = torch.arange(nv, device=device, dtype=torch.float64) - 0.5 * (nv - 1)
    for k0 in range(0, len(theta), 32):
        th = torch.as_tensor(theta[k0:k0 + 32], device=device, dtype=torch.float64)
        zz = torch.as_tensor(z[k0:k0 + 32], device=device, dtype=torch.float64)
        c, s = torch.cos(th), torch.sin(th)
        src = torch.stack([src_axis * c, src_axis * s, zz], 1)
        dcen = src + src_det * torch.stack([-c, -s, torch.zeros_like(c)], 1)
        eu = torch.stack([-s, c, torch.zeros_like(c)], 1)
        p = (dcen[:, None, None, :] + (ju[None, None, :, None] * pitch) * eu[:, None, None, :])
        p = p.expand(-1, nv, -1, -1).clone()
        p[..., 2] = p[..., 2] + (jv[None, :, None] * pitch)
        w = p - src[:, None, None, :]
        ax = (w[..., 1].abs() > w[..., 0].abs()).long()
        wa = torch.where(ax == 1, w[..., 1], w[..., 0])
        wb = torch.where(ax == 1, w[..., 0], w[..., 1])
        sa = torch.where(ax == 1, src[:, 1, None, None], src[:, 0, None, None]).expand_as(wa) / h + ic
        sb = torch.where(ax == 1, src[:, 0, None, None], src[:, 1, None, None]).expand_as(wa) / h + ic
        sz = (src[:, 2, None, None] / h + ic).expand_as(wa)
        lo = torch.zeros_like(wa)
        hi = torch.full_like(wa, n - 1.0)
        for (s0, wq) in ((sb, wb), (sz, w[..., 2])):
            r = wq / wa
            t1 = sa + (-1.0 - s0) / r
            t2 = sa + (n - s0) / r
            lo = torch.maximum(lo, torch.minimum(t1, t2))
            hi = torch.minimum(hi, torch.maximum(t1, t2))
        cnt = (torch.floor(hi) - torch.ceil(lo) + 1).clamp(min=0)
        total += float(cnt.sum())
    return 4.0 * total


# ---------------------------------------------------------------------------
# workload synthesis (GPU, torch + the library's projector)
# ---------------------------------------------------------------------------
def make_workload(name, device="cuda"):
    import torch
    from paper_2103_10329_gb300 import mgct, synth
    w = WORKLOADS[name]
    n, nu, K, L = w["n"], w["nu"], w["views"], w["levels"]
    th, z = synth.trajectory(K, SEED + 1)
    pitch = synth.default_pitch(nu)
    ph = synth.ellipsoids(w["count"], SEED, axis_lo=w["axis"][0], axis_hi=w["axis"][1])
    truth = synth.voxelize_ellipsoids(ph, n, supersample=2, device=device, dtype=torch.float32)
    tex = synth.porous_texture(n, SEED + 3, device=device) if w["texture"] else None
    if tex is not None:
        truth += tex
    if w["fine"] == 2:
        # data from a phantom twice as fine (no inverse crime)
        fine = synth.voxelize_ellipsoids(ph, 2 * n, supersample=1, device=device, dtype=torch.float32)
        if tex is not None:
            fine += tex.repeat_interleave(2, 0).repeat_interleave(2, 1).repeat_interleave(2, 2)
        gf = mgct.Geometry(2 * n, nu, nu, th, z, pitch, levels=1)
        b = mgct.project(gf, fine)
        del fine
        gf.close()
    else:
        # at 1024^3 a 2048^3 phantom and its projector copies would take about
        # 170 GB: the data come from the reconstruction grid's own phantom
        gf = mgct.Geometry(n, nu, nu, th, z, pitch, levels=1)
        b = mgct.project(gf, truth)
        gf.close()
    if w["photons"]:
        b = synth.poisson_log_data(b, w["photons"], SEED + 2)
    torch.cuda.synchronize()
    g = mgct.Geometry(n, nu, nu, th, z, pitch, levels=L)
    return dict(geom=g, b=b.contiguous(), truth=truth, theta=th, z=z, pitch=pitch, n=n, nu=nu, views=K,
                levels=L)


def train_correction(phantoms: int, steps: int, kernel=None):
    """The learned correction, trained on the GPU by the library's own kernels
    on pairs the method generates on random 128^3 phantoms (192^2 detector,
    360 views, 2 grids, 20 ellipsoids each).  With `kernel` (a 3x3x3
    preconditioner in place of Eq. 5, set on every training geometry) the
    network learns to correct that kernel's step instead."""
    import torch
    from paper_2103_10329_gb300 import learned as LN
    from paper_2103_10329_gb300 import mgct
    t0 = time.perf_counter()
    cases = [LN.make_case(128, 192, 360, 2, seed=20000 + i, count=20) for i in range(phantoms)]
    if kernel is not None:
        for geom, _, _ in cases:
            geom.set_preconditioner(kernel)
    pairs = LN.generate_pairs(cases, iters=2)
    for geom, _, _ in cases:
        geom.close()
    del cases
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net = mgct.Net(seed=0)
    hist = LN.train(net, pairs, steps=steps, crop=64, batch=4, lr=1e-3, log_every=max(1, steps // 10))
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del pairs
    return net, {"phantoms": phantoms, "pairs": 2 * phantoms, "steps": steps, "crop": 64, "batch": 4,
                 "pair_generation_s": t1 - t0, "training_s": t2 - t1, "loss_log": hist,
                 "config": "128^3, 192^2 detector, 360 views, 2 grids, 20 ellipsoids; Adam lr 1e-3, x0.3 after 70 %"}


def roi_rmse(vol, truth):
    import torch
    n = truth.shape[0]
    c = (torch.arange(n, device=truth.device, dtype=torch.float32) - (n - 1) / 2) / n
    r2 = c[None, :, None] ** 2 + c[None, None, :] ** 2
    m = (r2 <= (0.45) ** 2) & (c.abs()[:, None, None] <= 0.45)
    d = (vol - truth)[m]
    rng = float(truth.max() - truth.min())
    return float(torch.sqrt(torch.mean(d.double() ** 2))) / rng


# ---------------------------------------------------------------------------
# the oracle on host cores (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample(name, target_s=15.0, vol=None, views_cap=None, dims=None):
    """A and A^T of the FP64 oracle at grid 0 on a sample of views; returns
    (GUPS, seconds, views used, threads, seconds of A, seconds of A^T).
    `dims` = (n, detector, views) overrides the workload's sizes."""
    import oracle as O
    from paper_2103_10329_gb300 import synth
    if dims is None:
        w = WORKLOADS[name]
        n, nu, K = w["n"], w["nu"], w["views"]
    else:
        n, nu, K = dims
    th, z = synth.trajectory(K, SEED + 1)
    scan = O.Scan(n=n, nu=nu, nv=nu, theta=th, z=z, pitch=synth.default_pitch(nu))
    g = O.level_geometry(scan, 0)
    if vol is None:
        vol = synth.random_volume(n, SEED)
    if n >= 1024:
        return _oracle_sample_rows(g, vol, K)

    def run(cnt):
        gs = g.subset(np.arange(cnt))
        t0 = time.perf_counter()
        y = O.project(gs, vol)
        t1 = time.perf_counter()
        O.backproject(gs, y)
        t2 = time.perf_counter()
        return t2 - t0, t1 - t0, t2 - t1

    cnt = min(4, K)
    t = run(cnt)[0]
    if views_cap is None:
        cnt2 = int(max(cnt, min(K, cnt * target_s / max(t, 1e-3))))
    else:
        cnt2 = min(views_cap, K)
    t, ta, tat = run(cnt2)
    gups = 2.0 * n ** 3 * cnt2 / t / 1e9
    return gups, t, cnt2, O.num_threads(), ta, tat


ROW_SAMPLE = 16


def _oracle_sample_rows(g, vol, K):
    """The oracle at 1024^3, where its scatter A^T keeps one private FP64
    volume per thread within 8 GB and so runs on one thread: A over one whole
    view (all host threads), and A^T of that view on ROW_SAMPLE detector rows
    spread evenly over it (a sub-detector of every (nv / ROW_SAMPLE)-th row),
    scaled to the whole view by the row count.  Returns the tuple of
    oracle_sample with the view's A and A^T seconds."""
    import oracle as O
    k = K // 2
    gk = g.subset([k])
    step = max(1, g.nv // ROW_SAMPLE)
    r0 = (g.nv - step * (ROW_SAMPLE - 1)) // 2
    band = O.LevelGeom(g.n, g.nu, ROW_SAMPLE, g.h, gk.src, gk.det + r0 * gk.pv, gk.pu, step * gk.pv)
    t0 = time.perf_counter()
    O.project(gk, vol)
    t1 = time.perf_counter()
    yb = O.project(band, vol)
    t2 = time.perf_counter()
    O.backproject(band, yb)
    t3 = time.perf_counter()
    ta, tat = t1 - t0, (t3 - t2) * g.nv / ROW_SAMPLE
    gups = 2.0 * g.n ** 3 / (ta + tat) / 1e9
    return gups, (t1 - t0) + (t3 - t2), 1, O.num_threads(), ta, tat


def reference_arm(args, rank):
    if rank != 0:
        return
    name = args.workload
    w = WORKLOADS[name]
    import oracle as O
    O.build()
    from paper_2103_10329_gb300 import synth
    vol = synth.random_volume(w["n"], SEED)
    # one step = oracle A + A^T on a fixed sample of views (at 1024^3: one
    # view's A and A^T on a sample of its rows, scaled to the view)
    per_step_views = args.ref_views if w["n"] < 1024 else 1
    vals = []
    for i in range(args.warmup + args.steps):
        gups, t, cnt, thr, ta, tat = oracle_sample(name, vol=vol, views_cap=per_step_views)
        if i >= args.warmup:
            vals.append((gups, ta + tat))
    tot_t = sum(t for _, t in vals)
    units = 2.0 * w["n"] ** 3 * per_step_views * len(vals)
    value = units / tot_t / 1e9
    sample = (f"FP64 oracle A and A^T at grid 0 on {per_step_views} of {w['views']} views per step"
              if w["n"] < 1024 else
              f"FP64 oracle per step: A over one of {w['views']} views (all threads) and its A^T on "
              f"{ROW_SAMPLE} of {w['nu']} detector rows (one thread: 8 GB cap on the oracle's private "
              f"volumes), scaled to the view")
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(name),
            "cpu_baseline": {"value": value, "unit": "GUPS", "cores": thr, "host_cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _event_ms(fn, reps, warm=1):
    """Median CUDA-event time (ms) of fn() on the current stream."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(warm):
        fn()
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def _oracle_solve_units(n, views, levels, iters=2):
    """Voxel-view counts of the oracle's A and A^T calls in `iters` multigrid
    iterations: Landweber on grids 0..L-2 takes two A (residual, line search)
    and one A^T; its OS-EMTR pass on the coarsest grid takes two A (P 1 and the
    subsets' forward projections) and two A^T (numerator, denominator)."""
    ua = uat = 0
    for g in range(levels):
        u = (n >> g) ** 3 * views
        if levels == 1 or g < levels - 1:
            ua, uat = ua + 2 * u, uat + u
        else:
            ua, uat = ua + 2 * u, uat + 2 * u
    return iters * ua, iters * uat


def _ray_voxel_rates(og, vol, samples, sino_views=8):
    """Oracle seconds per ray of A and per voxel-view of A^T, from `samples`
    random rays (project_rays on `vol`) and random voxels over `sino_views`
    views (backproject_voxels on a random sinogram)."""
    import oracle as O
    from paper_2103_10329_gb300 import synth
    K = og.n_views
    rays = synth.random_indices(samples, (K, og.nv, og.nu), SEED + 11)
    t0 = time.perf_counter()
    O.project_rays(og, vol, rays)
    t_ray = (time.perf_counter() - t0) / samples
    sub = og.subset(np.arange(0, K, max(1, K // sino_views))[:sino_views])
    y = synth.random_sino(sub.n_views, og.nv, og.nu, SEED + 12)
    vox = synth.random_indices(samples, (og.n,) * 3, SEED + 13)
    t0 = time.perf_counter()
    O.backproject_voxels(sub, y, vox, radius=5)
    t_vox = (time.perf_counter() - t0) / (samples * sub.n_views)
    return t_ray, t_vox


def oracle_beside(c2_sample, c2_gpu, full_c2=False, samples=100000):
    """The FP64 oracle timed beside the GPU, on the host cores, per operation
    (one A and one A^T over every view, at grid 0) and per solve (two multigrid
    iterations from zero):
      64^3 / 96^2 / 90 views / 2 grids   both sides measured in full;
      256^3 / 384^2 / 720 views / 3 grids  oracle A and A^T on a sample of
          views scaled to all views (exact: views are independent), its solve
          extrapolated from those rates (measured in full with full_c2);
      512^3 / 768^2 / 1440 views          oracle on a sample of views;
      1024^3 / 1536^2 / 2880 views        oracle extrapolated by its per-nonzero
          rate at 512^3.
    Beside each view sample, the time extrapolated from random rays
    (project_rays) and random voxels (backproject_voxels) is reported as a
    check: the per-voxel routine evaluates the per-entry weight over a pixel
    window, far slower than the oracle's scatter A^T, so those rates do not
    stand for the whole calls.  GPU times are CUDA-event medians of the
    library's public calls."""
    import torch
    import oracle as O
    from paper_2103_10329_gb300 import mgct, synth
    out = {"threads": O.num_threads(), "host_cores": len(os.sched_getaffinity(0)),
           "timing": "oracle: wall clock, FP64, all host threads; GPU: CUDA events, FP32, median", "configs": {}}

    def scan_of(n, nu, K):
        th, z = synth.trajectory(K, SEED + 1)
        return O.Scan(n=n, nu=nu, nv=nu, theta=th, z=z, pitch=synth.default_pitch(nu)), th, z

    def per_op(o_a, o_at, g_a, g_at, how):
        return {"A": {"oracle_s": o_a, "gpu_ms": g_a, "speedup": o_a * 1e3 / g_a},
                "AT": {"oracle_s": o_at, "gpu_ms": g_at, "speedup": o_at * 1e3 / g_at}, "oracle": how}

    def gpu_ops(g, vol, reps, warm=1):
        y = mgct.project(g, vol)
        t_a = _event_ms(lambda: mgct.project(g, vol, out=y), reps, warm)
        vo = torch.empty_like(vol)
        t_at = _event_ms(lambda: mgct.backproject(g, y, out=vo), reps, warm)
        return t_a, t_at

    def gpu_solve(g, b, reps=3):
        rec = mgct.Reconstructor(g)
        rec.prepare(b)
        n = g.n
        v = torch.zeros((n, n, n), device="cuda")

        def run():
            v.zero_()
            rec.iterate(v)
            rec.iterate(v)
        t = _event_ms(run, reps)
        return t, v

    # --- 64^3: everything measured on both sides
    w = WORKLOADS["c1"]
    n, nu, K, L = w["n"], w["nu"], w["views"], w["levels"]
    W = make_workload("c1")
    g, b, truth = W["geom"], W["b"], W["truth"]
    vol = synth.random_volume(n, SEED)
    ga, gat = gpu_ops(g, torch.as_tensor(vol, dtype=torch.float32, device="cuda"), 10, 3)
    scan, th, z = scan_of(n, nu, K)
    og = O.level_geometry(scan, 0)
    ta = min(_timed(lambda: O.project(og, vol)) for _ in range(3))
    y = O.project(og, vol)
    tat = min(_timed(lambda: O.backproject(og, y)) for _ in range(3))
    gs_ms, vg = gpu_solve(g, b)
    ph = synth.ellipsoids(w["count"], SEED, axis_lo=w["axis"][0], axis_hi=w["axis"][1])
    fine = synth.voxelize_ellipsoids(ph, 2 * n, supersample=1, device="cpu", dtype=torch.float64).numpy()
    b_or = O.project(O.level_geometry(scan_of(2 * n, nu, K)[0], 0), fine)
    t0 = time.perf_counter()
    vo = O.reconstruct(scan, b_or, iters=2, levels=L)
    ts = time.perf_counter() - t0
    ua, uat = _oracle_solve_units(n, K, L)
    ext = ua * ta / (n ** 3 * K) + uat * tat / (n ** 3 * K)
    out["configs"]["64^3/96^2/90 views/2 grids"] = {
        "per_op": per_op(ta, tat, ga, gat, "measured, whole call (best of 3)"),
        "per_solve": {"oracle_s": ts, "gpu_ms": gs_ms, "speedup": ts * 1e3 / gs_ms, "oracle": "measured",
                      "oracle_extrapolated_s": ext,
                      "rmse_roi": {"oracle": roi_rmse(torch.from_numpy(vo).float(), truth.cpu()),
                                   "gpu": roi_rmse(vg, truth)},
                      "data": "each side projects the same 128^3 phantom with its own A"}}
    g.close()
    del W, b, truth, vg

    # --- the bench workload: oracle per-op from the view sample of the CPU baseline
    w = WORKLOADS["c2"]
    n, nu, K, L = w["n"], w["nu"], w["views"], w["levels"]
    cnt, s_a, s_at, vol2 = c2_sample
    ta, tat = s_a * K / cnt, s_at * K / cnt
    g, b = c2_gpu
    ga, gat = gpu_ops(g, torch.as_tensor(vol2, dtype=torch.float32, device="cuda"), 3)
    gs_ms, _ = gpu_solve(g, b)
    scan, th, z = scan_of(n, nu, K)
    og = O.level_geometry(scan, 0)
    r_ray, r_vox = _ray_voxel_rates(og, vol2, samples)
    ua, uat = _oracle_solve_units(n, K, L)
    solve = {"gpu_ms": gs_ms, "oracle_extrapolated_s": ua * ta / (n ** 3 * K) + uat * tat / (n ** 3 * K)}
    if full_c2:
        b_or = O.project(og, vol2)
        t0 = time.perf_counter()
        O.reconstruct(scan, b_or, iters=2, levels=L)
        solve["oracle_s"] = time.perf_counter() - t0
        solve["oracle"] = "measured on b = A x (the oracle's A; solve time does not depend on the data)"
    else:
        solve["oracle"] = "extrapolated from the per-operation rates (A and A^T calls only)"
    solve["speedup"] = solve.get("oracle_s", solve["oracle_extrapolated_s"]) * 1e3 / gs_ms
    rays_ext = {"A_s": r_ray * K * nu * nu, "AT_s": r_vox * n ** 3 * K}
    out["configs"]["256^3/384^2/720 views/3 grids"] = {
        "per_op": per_op(ta, tat, ga, gat, f"measured on {cnt} of {K} views, scaled to all views"),
        "per_solve": solve, "ray_voxel_extrapolation_check": rays_ext}

    # --- 512^3: oracle on a sample of views, GPU whole calls
    n, nu, K = 512, 768, 1440
    vol = synth.random_volume(n, SEED)
    _, _, cnt, _, s_a, s_at = oracle_sample(None, target_s=8.0, vol=vol, dims=(n, nu, K))
    ta, tat = s_a * K / cnt, s_at * K / cnt
    scan, th, z = scan_of(n, nu, K)
    og = O.level_geometry(scan, 0)
    r_ray, r_vox = _ray_voxel_rates(og, vol, samples)
    g = mgct.Geometry(n, nu, nu, th, z, synth.default_pitch(nu), levels=1)
    ga, gat = gpu_ops(g, torch.as_tensor(vol, dtype=torch.float32, device="cuda"), 3)
    g.close()
    del vol
    torch.cuda.empty_cache()
    out["configs"]["512^3/768^2/1440 views"] = {
        "per_op": per_op(ta, tat, ga, gat, f"measured on {cnt} of {K} views, scaled to all views"),
        "ray_voxel_extrapolation_check": {"A_s": r_ray * K * nu * nu, "AT_s": r_vox * n ** 3 * K}}
    nnz3, ta3, tat3 = K * nu * nu * n, ta, tat

    # --- 1024^3: oracle extrapolated by its per-nonzero rate at 512^3; GPU whole calls
    n, nu, K = 1024, 1536, 2880
    scan, th, z = scan_of(n, nu, K)
    og = O.level_geometry(scan, 0)
    vol = np.full((n, n, n), 0.5)
    r_ray, r_vox = _ray_voxel_rates(og, vol, samples)
    del vol
    g = mgct.Geometry(n, nu, nu, th, z, synth.default_pitch(nu), levels=1)
    gv = torch.full((n, n, n), 0.5, device="cuda")
    y = torch.empty((K, nu, nu), device="cuda")
    mgct.project(g, gv, views=(0, 1, 1), out=y[:1])
    ga = _event_ms(lambda: mgct.project(g, gv, out=y), 1, 0)
    mgct.backproject(g, y[:1].contiguous(), views=(0, 1, 1))
    gat = _event_ms(lambda: mgct.backproject(g, y, out=gv), 1, 0)
    g.close()
    del gv, y
    torch.cuda.empty_cache()
    f = K * nu * nu * n / nnz3
    out["configs"]["1024^3/1536^2/2880 views"] = {
        "per_op": per_op(ta3 * f, tat3 * f, ga, gat,
                         f"extrapolated by the per-nonzero rate measured at 512^3 (nonzeros of A grow as "
                         f"views x pixels x n: {f:.0f}x)"),
        "ray_voxel_extrapolation_check": {"A_s": r_ray * K * nu * nu, "AT_s": r_vox * n ** 3 * K},
        "volume": "constant 0.5 on both sides"}
    return out


def _timed(fn):
    t0 = time.perf_counter()
    fn()
    return time.perf_counter() - t0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def traffic_record(kernel):
    """ncu DRAM bytes per launch recorded in profiles/traffic.json, if the
    kernel sources are unchanged since the capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        rec = json.load(open(p)).get(kernel)
        if not rec:
            return None
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() != rec["sha256"]:
            return None
        return rec
    except Exception:
        return None


def literal_tta(rec, g, truth, net, workload=None, target=1e-3, cap=50):
    """Seconds until RMSE_ROI <= 1e-3 on inverse-crime data (b = A truth,
    this library's A on the reconstruction grid, no noise), per form, capped
    at `cap` multigrid iterations; "not reached" with the last RMSE otherwise.
    With `workload`, the geometry and phantom are that workload's."""
    import torch
    from paper_2103_10329_gb300 import mgct
    own = workload is not None
    if own:
        W = make_workload(workload)
        g, truth = W["geom"], W["truth"]
        rec = mgct.Reconstructor(g)
    b_ic = mgct.project(g, truth)
    rec.prepare(b_ic)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    forms = [("fp32", torch.float32, None, False), ("bf16", torch.bfloat16, None, False),
             ("fp32_fas", torch.float32, None, True), ("bf16_fas", torch.bfloat16, None, True),
             ("bf16_fas_fp32_every_4th", "refresh4", None, True),
             ("bf16_fas_fp32_every_2nd", "refresh2", None, True), ("fp16_fas", torch.float16, None, True)]
    if net is not None:
        forms += [("learned_bf16", torch.bfloat16, net, False), ("learned_bf16_fas", torch.bfloat16, net, True)]
    out = {"data": "inverse crime: b = A truth (this library's A on the reconstruction grid), no noise",
           "fas": "the *_fas forms take the full-approximation-scheme coarse data R(b - A mu) + A_c R mu "
                  "(a variant outside the paper; one extra A per grid per iteration)",
           "target_rmse_roi": target, "cap_iters": cap, "forms": {}}
    for name, st, nn, fas in forms:
        v = torch.zeros_like(truth)
        tot, rm, it = 0.0, None, 0
        for it in range(1, cap + 1):
            torch.cuda.synchronize()
            s0.record()
            if isinstance(st, str):
                # BF16 copies of mu round at about 1e-3 of its range, the
                # target itself; one float32 iteration in every k lowers the floor
                k = int(st[len("refresh"):])
                rec.iterate(v, storage=torch.float32 if it % k == 0 else torch.bfloat16, fas=fas)
            elif nn is None:
                rec.iterate(v, storage=st, fas=fas)
            else:
                rec.iterate_learned(v, nn, storage=st, fas=fas)
            s1.record()
            torch.cuda.synchronize()
            tot += s0.elapsed_time(s1)
            rm = roi_rmse(v, truth)
            if rm <= target:
                break
        reached = rm is not None and rm <= target
        out["forms"][name] = {"reached": reached, "iters": it if reached else None,
                              "seconds": tot / 1e3 if reached else None,
                              "last_rmse_roi": rm, "iters_run": it, "ms_run": tot}
    if own:
        g.close()
    return out


def hbm_kernel_rates(peak_gbs, n=512, reps=5):
    """The HBM-bound kernels of the step, each through the C ABI on arrays
    larger than L2 (512^3 float32 = 537 MB): achieved GB/s from algorithmic
    bytes (each array read or written once) over the CUDA-event time of one
    launch (median of `reps`, after two warm-up launches)."""
    import torch
    from paper_2103_10329_gb300 import mgct, synth
    dev = "cuda"
    g = torch.Generator(device=dev).manual_seed(1)
    x = torch.rand((n, n, n), device=dev, generator=g)
    y = torch.rand((n, n, n), device=dev, generator=g)
    o = torch.empty_like(x)
    c1 = torch.rand((n // 2,) * 3, device=dev, generator=g)
    c0 = torch.rand((n // 2,) * 3, device=dev, generator=g)
    kv, nvs = 360, 2 * n  # a sinogram of 360 views of (2n)^2 pixels: 1.5 GB
    sino = torch.rand((kv, nvs, nvs), device=dev, generator=g)
    th, z = synth.trajectory(2, 1)
    geom = mgct.Geometry(n, 16, 16, th, z, synth.default_pitch(16), levels=1)
    vox = n ** 3
    cases = {
        "precondition (Eq. 5 stencil)": (lambda: mgct.precondition(geom, x, out=o), 8.0 * vox),
        "update y += a x": (lambda: mgct.axpy(0.5, x, y), 12.0 * vox),
        "restrict_volume (2x2x2 mean)": (lambda: mgct.restrict_volume(x, out=c1), 4.5 * vox),
        "prolong_add (trilinear)": (lambda: mgct.prolong_add(c1, c0, y), 9.0 * vox),
        "restrict_sino (2x2 mean)": (lambda: mgct.restrict_sino(sino), 5.0 * kv * nvs * nvs),
    }
    out = {}
    for name, (fn, nbytes) in cases.items():
        for _ in range(2):
            fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = sorted(ts)[len(ts) // 2]
        gbs = nbytes / (ms / 1e3) / 1e9
        out[name] = {"ms": ms, "bytes_alg": nbytes, "gbs": gbs, "frac_of_measured_hbm": gbs / peak_gbs}
    geom.close()
    return {"size": f"{n}^3 volumes (537 MB, larger than L2), sinogram {kv} x {nvs}^2", "peak_gbs": peak_gbs,
            "kernels": out}


def time_to_accuracy(args, W, rec, g, b, truth, vol):
    """On the 256^3 / 720-view workload: PMGL vs SIRT at equal fine-grid
    cost (FP32), full-resolution OS-EMTR, the 16-bit storage forms, the
    learned correction (trained here), the BilateralFilter and PSF-kernel
    forms against the plain FP32 two-iteration RMSE E2, and the literal
    RMSE <= 1e-3 clock."""
    import torch
    from paper_2103_10329_gb300 import mgct
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)

    def run_iters(storage, iters, net=None, bilateral=None, learned_iters=None):
        """Per-iteration (cumulative ms, RMSE_ROI); with `net`, the learned
        step on the first `learned_iters` iterations (all when None), the
        plain one after (the gate)."""
        v = torch.zeros_like(vol)
        out = []
        tot = 0.0
        for it in range(iters):
            torch.cuda.synchronize()
            s0.record()
            if net is None or (learned_iters is not None and it >= learned_iters):
                rec.iterate(v, storage=storage, bilateral=bilateral)
            else:
                rec.iterate_learned(v, net, storage=storage)
            s1.record()
            torch.cuda.synchronize()
            tot += s0.elapsed_time(s1)
            out.append((tot, roi_rmse(v, truth)))
        return out

    base = run_iters(torch.float32, 2)
    e2 = base[-1][1]
    vs = torch.zeros_like(vol)
    ws = mgct.workspace(g, mgct.WS_LANDWEBER, 0)
    s0.record()
    for _ in range(2):
        mgct.landweber_step(g, vs, b, precond=False, ws=ws)
    s1.record()
    torch.cuda.synchronize()
    tta = {"rmse_def": "RMS(mu - truth) / range(truth) over r <= 0.9R, |z| <= 0.9R",
           "E2_pmgl_fp32_2iter": e2, "pmgl_fp32_2iter_ms": base[-1][0],
           "sirt_2iter_ms": s0.elapsed_time(s1), "sirt_2iter_rmse_roi": roi_rmse(vs, truth),
           "forms": {}}
    # Fig. 2 analogue: OS-EMTR (Eq. 3, M = 8 subsets) at full resolution
    del vs
    ones = torch.ones_like(vol)
    pi = mgct.project(g, ones)
    del ones
    we = mgct.workspace(g, mgct.WS_OSEMTR, 0)
    ve = torch.zeros_like(vol)
    em, tot = [], 0.0
    for _ in range(10):
        torch.cuda.synchronize()
        s0.record()
        mgct.osemtr_pass(g, ve, b, pi, n_subsets=8, ws=we)
        s1.record()
        torch.cuda.synchronize()
        tot += s0.elapsed_time(s1)
        em.append((tot, roi_rmse(ve, truth)))
    tta["osemtr_full_res"] = {"subsets": 8, "per_pass_ms_cum": [e[0] for e in em],
                              "per_pass_rmse_roi": [e[1] for e in em]}
    del ve, we, pi
    net = None
    if not args.no_learned:
        t0 = time.perf_counter()
        net, train_info = train_correction(args.learn_phantoms, args.learn_steps)
        train_info["wall_s"] = time.perf_counter() - t0
        tta["learned_training"] = train_info
    forms = [("fp32", torch.float32, False), ("bf16", torch.bfloat16, False), ("fp16", torch.float16, False)]
    if net is not None:
        forms += [("learned_fp32", torch.float32, True), ("learned_bf16", torch.bfloat16, True)]
    # Alg. 1's BilateralFilter (no parameters in the paper): sigma_s = 1 voxel,
    # sigma_r = 0.2, radius 1, the best of five settings tried on this workload
    bil = (1.0, 0.2, 1)
    forms += [("bilateral_fp32", torch.float32, "bil"), ("bilateral_bf16", torch.bfloat16, "bil")]
    tta["bilateral"] = {"sigma_s_voxels": bil[0], "sigma_r": bil[1], "radius": bil[2],
                        "chosen": "best of (1, 0.05, 1), (1, 0.1, 1), (1, 0.2, 1), (1.5, 0.1, 2), (0.8, 0.1, 1) "
                                  "on this workload; E2 stays the plain form's"}
    # a preconditioner fitted to the measured PSF of A^T A (in place of Eq. 5)
    from paper_2103_10329_gb300 import psf as PSF
    t0 = time.perf_counter()
    kern, _ = PSF.derived_preconditioner(g)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    g.set_preconditioner(kern)
    hist_psf = run_iters(torch.float32, 3)
    g.set_preconditioner(None)
    reach = next(((i + 1, t) for i, (t, e) in enumerate(hist_psf) if e <= e2 * (1 + 1e-3)), None)
    tta["forms"]["psf_kernel_fp32"] = {"per_iter_ms_cum": [h[0] for h in hist_psf],
                                       "per_iter_rmse_roi": [h[1] for h in hist_psf],
                                       "iters_to_E2": reach[0] if reach else None,
                                       "ms_to_E2": reach[1] if reach else None}
    tta["psf_kernel"] = {"kernel_z0_plane": kern[1].tolist(), "kernel_z1_plane": kern[2].tolist(),
                         "measure_and_fit_s": fit_s,
                         "per_iter_ms_cum": [h[0] for h in hist_psf], "per_iter_rmse_roi": [h[1] for h in hist_psf]}
    for name, st, use_net in forms:
        if use_net == "bil":
            hist = run_iters(st, 3, None, bil)
        else:
            hist = run_iters(st, 3, net if use_net else None)
        reach = next(((i + 1, t) for i, (t, e) in enumerate(hist) if e <= e2 * (1 + 1e-3)), None)
        tta["forms"][name] = {"per_iter_ms_cum": [h[0] for h in hist], "per_iter_rmse_roi": [h[1] for h in hist],
                              "iters_to_E2": reach[0] if reach else None,
                              "ms_to_E2": reach[1] if reach else None}
    if net is not None:
        # the gate: the correction on the first iteration only (it gains early
        # and hurts late), plain Alg. 1 after
        hist = run_iters(torch.bfloat16, 3, net, learned_iters=1)
        reach = next(((i + 1, t) for i, (t, e) in enumerate(hist) if e <= e2 * (1 + 1e-3)), None)
        tta["forms"]["learned_bf16_first_iteration_only"] = {
            "per_iter_ms_cum": [h[0] for h in hist], "per_iter_rmse_roi": [h[1] for h in hist],
            "iters_to_E2": reach[0] if reach else None, "ms_to_E2": reach[1] if reach else None}
    if not args.no_learned:
        # the correction trained on top of the PSF-derived kernel, against that
        # kernel's own two-iteration RMSE E_psf2 (which one plain iteration of
        # it does not reach)
        t0 = time.perf_counter()
        net_psf, info_psf = train_correction(args.learn_phantoms, args.learn_steps, kernel=kern)
        info_psf["wall_s"] = time.perf_counter() - t0
        tta["learned_psf_training"] = info_psf
        e_psf2 = hist_psf[1][1]
        g.set_preconditioner(kern)
        tta["E_psf2"] = e_psf2
        for name, st, nn_, li in (("psf_kernel_fp32", torch.float32, None, None),
                                  ("learned_psf_fp32", torch.float32, net_psf, None),
                                  ("learned_psf_bf16", torch.bfloat16, net_psf, None),
                                  ("learned_psf_bf16_first_iteration_only", torch.bfloat16, net_psf, 1)):
            hist = run_iters(st, 3, nn_, learned_iters=li)
            r2 = next(((i + 1, t) for i, (t, e) in enumerate(hist) if e <= e2 * (1 + 1e-3)), None)
            rp = next(((i + 1, t) for i, (t, e) in enumerate(hist) if e <= e_psf2 * (1 + 1e-3)), None)
            tta.setdefault("psf_forms", {})[name] = {
                "per_iter_ms_cum": [h[0] for h in hist], "per_iter_rmse_roi": [h[1] for h in hist],
                "ms_to_E2": r2[1] if r2 else None, "ms_to_E_psf2": rp[1] if rp else None,
                "iters_to_E_psf2": rp[0] if rp else None}
        g.set_preconditioner(None)
        net_psf.close()
    tta["E2_tolerance"] = "RMSE <= E2 (1 + 1e-3)"
    if not args.no_literal:
        tta["literal_rmse_1e-3"] = {
            "c2": literal_tta(rec, g, truth, net),
            "c1": literal_tta(None, None, None, net, workload="c1"),
        }
        rec.prepare(b)

    return tta


def joint_estimation_c4(seed=SEED + 4, schedule=((2, 2), (1, 2), (0, 2)), mg_iters=2, **step_kw):
    """The drift workload: 256^3 phantom (200 ellipsoids + porous texture, no
    noise), 384^2 detector, 720 views, every view's source and detector
    offsets and detector tilt drifting as Gaussian random walks of 0.3 px per
    view; data projected from the 2x finer phantom under the true drift.
    Joint estimation (joint.estimate) from no drift; reported: the drift RMSE
    per parameter type, the projection shifts of the volume centre, and the
    image RMSE (ROI) against the phantom for no correction, the estimated
    drift and the true drift, each after the same number of multigrid
    iterations."""
    import torch
    from paper_2103_10329_gb300 import joint, mgct, synth
    w = WORKLOADS["c2"]
    n, nu, K = w["n"], w["nu"], w["views"]
    th, z = synth.trajectory(K, SEED + 1)
    pitch = synth.default_pitch(nu)
    half = 0.5 * math.sqrt(2.0) * nu
    true = synth.drift_walk(K, seed, sigma_px=0.3, half_diag_px=half)
    ph = synth.ellipsoids(w["count"], SEED, axis_lo=w["axis"][0], axis_hi=w["axis"][1])
    truth = synth.voxelize_ellipsoids(ph, n, supersample=2, device="cuda", dtype=torch.float32)
    tex = synth.porous_texture(n, SEED + 3, device="cuda")
    truth += tex
    fine = synth.voxelize_ellipsoids(ph, 2 * n, supersample=1, device="cuda", dtype=torch.float32)
    fine += tex.repeat_interleave(2, 0).repeat_interleave(2, 1).repeat_interleave(2, 2)
    del tex
    gf = mgct.Geometry(2 * n, nu, nu, th, z, pitch, levels=1, drift=true)
    b = mgct.project(gf, fine)
    gf.close()
    del fine
    g = mgct.Geometry(n, nu, nu, th, z, pitch, levels=3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mu, phi, hist = joint.estimate(g, b, half, schedule=schedule, truth_phi=true, mg_iters=mg_iters, **step_kw)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    iters = mg_iters * (sum(r for _, r in schedule) + 1)
    rec = mgct.Reconstructor(g)

    def data_residual(p, v):
        g.set_drift(p)
        r = mgct.project(g, v, b=b)
        return float(torch.linalg.vector_norm(r.double()) / torch.linalg.vector_norm(b.double()))

    out_img = {"estimated": roi_rmse(mu, truth)}
    out_res = {"estimated": data_residual(phi, mu)}
    for name, p in (("no_correction", None), ("true_drift", true)):
        g.set_drift(p)
        rec.prepare(b)
        v = torch.zeros_like(mu)
        for _ in range(iters):
            rec.iterate(v)
        out_img[name] = roi_rmse(v, truth)
        out_res[name] = data_residual(p, v)
    g.close()
    err = phi - true
    rms = lambda a: np.sqrt(np.mean(a ** 2, axis=0)).tolist()
    # The data fix the drift only up to a rigid motion of the object: a
    # translation (ds_u = dd_u = a sin(theta) + b cos(theta) in-plane;
    # ds_v = dd_v = c vertically), a turn about z (ds_u = -dd_u = c) and about
    # a horizontal axis (ds_v = -dd_v = a sin(theta) + b cos(theta)), at the
    # source and detector distances 2 and 2 of this geometry.  The gauge-free
    # error removes the least-squares fit of those six fields.
    sn, cs, one = np.sin(th), np.cos(th), np.ones(K)
    zero = np.zeros(K)
    basis = []
    for f in (sn, cs):
        basis.append(np.stack([f, zero, f, zero, zero], 1))      # in-plane translation
        basis.append(np.stack([zero, f, zero, -f, zero], 1))     # turn about a horizontal axis
    basis.append(np.stack([zero, one, zero, one, zero], 1))      # vertical translation
    basis.append(np.stack([one, zero, -one, zero, zero], 1))     # turn about z
    Bm = np.stack([bb.ravel() for bb in basis], 1)
    coef, *_ = np.linalg.lstsq(Bm, err.ravel(), rcond=None)
    err_gf = err - (Bm @ coef).reshape(K, 5)
    coef0, *_ = np.linalg.lstsq(Bm, true.ravel(), rcond=None)
    true_gf = true - (Bm @ coef0).reshape(K, 5)
    return {"workload": "256^3 (200 ellipsoids + porous texture, noise-free), 384^2 detector, 720 views, 3 grids; "
                        "drift: source and detector offsets and tilt as 0.3 px/view Gaussian random walks; data "
                        "from the 2x finer phantom under the true drift",
            "schedule": [list(s) for s in schedule], "multigrid_iterations": iters, "seconds": secs,
            "parameters": ["ds_u", "ds_v", "dd_u", "dd_v", "psi"],
            "drift_rmse": {"no_correction": rms(true), "estimated": rms(err)},
            "drift_rmse_gauge_free": {"no_correction": rms(true_gf), "estimated": rms(err_gf),
                                      "gauge": "rigid motions of the object removed (least-squares fit of "
                                               "six per-view fields)"},
            "relative_data_residual": out_res,
            "centre_shift_rmse_px": {"u (ds_u + dd_u)": {"no_correction": float(rms(true[:, 0] + true[:, 2])),
                                                          "estimated": float(rms(err[:, 0] + err[:, 2]))},
                                     "v (ds_v + dd_v)": {"no_correction": float(rms(true[:, 1] + true[:, 3])),
                                                          "estimated": float(rms(err[:, 1] + err[:, 3]))}},
            "image_rmse_roi": out_img, "history": hist}


def evaluation_1024(args):
    """The learned correction at the 1024^3 / 1536^2 / 2880-view evaluation
    size (the headline workload): two multigrid iterations from zero of the
    plain form (Eq. 5), the PSF-derived kernel, and the correction trained on
    top of that kernel (128^3 training phantoms, BF16 tensor-core network
    applied in z-slabs), each with its RMSE (ROI) per iteration and its
    seconds.  The kernel is fitted on the 256^3 / 720-view geometry of the
    same family (same distances and detector-to-voxel ratio): the fit's PSF
    measurement at 1024^3 would take several full A^T A applications."""
    import torch
    from paper_2103_10329_gb300 import mgct
    from paper_2103_10329_gb300 import psf as PSF
    w2 = WORKLOADS["c2"]
    from paper_2103_10329_gb300 import synth
    th2, z2 = synth.trajectory(w2["views"], SEED + 1)
    g2 = mgct.Geometry(w2["n"], w2["nu"], w2["nu"], th2, z2, synth.default_pitch(w2["nu"]), levels=w2["levels"])
    kern, _ = PSF.derived_preconditioner(g2)
    g2.close()
    t0 = time.perf_counter()
    net_psf, info = train_correction(args.learn_phantoms, args.learn_steps, kernel=kern)
    info["wall_s"] = time.perf_counter() - t0
    W = make_workload("c5")
    g, b, truth = W["geom"], W["b"], W["truth"]
    rec = mgct.Reconstructor(g)
    rec.prepare(b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": workload_config("c5")["workload"], "training": info, "forms": {}}
    for name, k, nn in (("plain_eq5", None, None), ("psf_kernel", kern, None), ("learned_on_psf_bf16", kern, net_psf)):
        g.set_preconditioner(k)
        v = torch.zeros_like(truth)
        hist = []
        tot = 0.0
        for _ in range(2):
            torch.cuda.synchronize()
            e0.record()
            if nn is None:
                rec.iterate(v)
            else:
                rec.iterate_learned(v, nn, storage=torch.bfloat16)
            e1.record()
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
            hist.append((tot / 1e3, roi_rmse(v, truth)))
        out["forms"][name] = {"seconds_cum": [h[0] for h in hist], "rmse_roi": [h[1] for h in hist]}
        del v
    g.set_preconditioner(None)
    net_psf.close()
    g.close()
    return out


def family_rooflines(W, nnz, trace0, peaks, sm_clock, fp32_peak, mp=None):
    """Roofline objects of the projector and back-projector families on the
    finest grid: one grid-0 launch is one A (or A^T) over every view.  The
    fraction is t_floor / t_launch with t_floor the largest of three floors
    per launch:
      HBM: one volume plus one sinogram at the measured copy bandwidth;
      on-chip gather: 4 B per nonzero of A against the L1 at 128 B/clk/SM
        (the binding floor of both families);
      FP32: 2 flop per nonzero plus ~8 per sample against 128 lanes/SM.
    `traffic` is the ncu DRAM bytes of the family's kernel recorded in
    profiles/traffic.json, per launch: measured on its own workload, scaled
    by the nonzeros from a smaller capture otherwise (stated in the object)."""
    n, K, nu = W["n"], W["views"], W["nu"]
    l1_peak = SMS * 128 * sm_clock * 1e6  # B/s
    hbm_b = 4 * (n ** 3 + K * nu ** 2)
    gather_b = 4 * nnz[0]
    fl = 2 * nnz[0] + 8 * (nnz[0] / 4)
    floors = {"hbm_ms": hbm_b / (peaks.get("hbm_gbs", 6790.0) * 1e9) * 1e3,
              "onchip_gather_ms": gather_b / l1_peak * 1e3,
              "fp32_ms": fl / (fp32_peak * 1e12) * 1e3}
    names = {"project": "k_project_col", "backproject": "k_backproject_reg"}
    out = {}
    for fam, kname in names.items():
        if fam not in trace0 or not trace0[fam][1]:
            continue
        t0_ms, t0_n = trace0[fam]
        avg_ms = t0_ms / max(t0_n, 1)
        t_s = avg_ms / 1e3
        tr = traffic_record(kname)
        traffic, tnote = None, None
        if tr:
            if tr.get("workload") == W["name"]:
                traffic, tnote = tr["bytes_per_launch"], f"ncu capture of this workload ({tr['how']})"
            elif tr.get("nnz_per_launch"):
                traffic = tr["bytes_per_launch"] * nnz[0] / tr["nnz_per_launch"]
                tnote = (f"scaled by nonzeros from the ncu capture at {tr.get('workload')} ({tr['how']}); "
                         "L2 reuse falls at larger volumes, so the true figure is higher")
        r = {"kernel": kname, "launches": "grid 0 (the finest grid)", "bound": "onchip-gather",
             "binding_floor": "on-chip gather (L1, 4 B per nonzero of A), the largest of the three floors",
             "achieved": gather_b / t_s / 1e9, "peak": l1_peak / 1e9, "unit": "GB/s",
             "frac": gather_b / t_s / l1_peak,
             "peak_source": f"derived: {SMS} SMs x 128 B/clk x {sm_clock:.0f} MHz of L1",
             "def": "frac = t_floor / t_launch, t_floor = max(HBM, on-chip gather, FP32 floors); achieved = "
                    "4 B per nonzero of A per launch / launch time",
             "floors_ms": floors, "avg_launch_ms": avg_ms, "launches_timed": t0_n,
             "work": f"{nnz[0]:.4g} nonzeros of A per launch (4 bilinear taps per in-volume sample)",
             "traffic": traffic, "traffic_note": tnote,
             "fp32": {"achieved_tflops": fl / t_s / 1e12, "peak_tflops": fp32_peak,
                      "frac": fl / t_s / 1e12 / fp32_peak},
             "hbm": {"bytes_alg": hbm_b, "frac_of_measured": hbm_b / t_s / 1e9 / peaks.get("hbm_gbs", 6790.0)}}
        if mp:
            r["measured_onchip"] = {"lds_gbs": mp["lds_gbs"], "fp32_tflops": mp["fp32_tflops"],
                                    "gather_frac_of_measured_lds": gather_b / t_s / 1e9 / mp["lds_gbs"]}
        out[kname] = r
    return out


def kernel_table(W, nnz, trace, steps):
    """Per-family time, launches, share, algorithmic TFLOP/s and GUPS per step."""
    n, K, L = W["n"], W["views"], W["levels"]
    flops = {"project": 0.0, "backproject": 0.0}
    for lv in range(L):
        if L == 1 or lv < L - 1:
            flops["project"] += 2 * 2 * nnz[lv]
            flops["backproject"] += 2 * nnz[lv]
        else:
            flops["project"] += 2 * nnz[lv]
            flops["backproject"] += 2 * 2 * nnz[lv]
    traced = sum(v[0] for v in trace.values() if v[1])
    kernels = {}
    for k, (t, c) in trace.items():
        if not c:
            continue
        e = {"ms_per_step": t / steps, "launches_per_step": c / steps, "share": t / traced}
        if k in flops:
            e["tflops_alg"] = flops[k] * steps / (t / 1e3) / 1e12
            vv = 0
            for lv in range(L):
                calls = (2 if k == "project" else 1) if (L == 1 or lv < L - 1) else 1
                vv += calls * (n >> lv) ** 3 * K
            e["gups"] = vv * steps / (t / 1e3) / 1e9
        kernels[k] = e
    return kernels


def time_steps(rec, vol, steps, warmup, barrier=lambda: None, clocks=None):
    """`warmup` untimed iterations, then `steps` timed ones between CUDA
    events (launch count and per-family trace taken over the timed ones)."""
    import torch
    from paper_2103_10329_gb300 import mgct
    for _ in range(warmup):
        rec.iterate(vol)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    mgct.trace_enable(True)
    mgct.launch_count(reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        rec.iterate(vol)
    ev1.record()
    torch.cuda.synchronize()
    launches = mgct.launch_count()
    barrier()
    ms = ev0.elapsed_time(ev1)
    trace = mgct.trace_read()
    trace0 = mgct.trace_read(level=0)
    mgct.trace_enable(False)
    clk = clocks.stop() if clocks else None
    return ms, launches, trace, trace0, clk


def gpu_arm(args, rank, world):
    import torch
    from paper_2103_10329_gb300 import build, mgct
    if world > 1:
        import torch.distributed as dist
    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    sm_clock = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * sm_clock * 1e6 / 1e12  # TFLOP/s
    try:
        mp = mgct.measure_onchip_peaks()
    except Exception:  # noqa: BLE001
        mp = None

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # ---- the headline workload, inputs resident on the device
    W = make_workload(args.workload)
    W["name"] = args.workload
    g, b, truth = W["geom"], W["b"], W["truth"]
    n, K, L = W["n"], W["views"], W["levels"]
    rec = mgct.Reconstructor(g)
    rec.prepare(b)
    vol = torch.zeros((n, n, n), device=dev, dtype=torch.float32)
    units = units_per_step(n, K, L)
    ms, launches, trace, trace0, clk = time_steps(rec, vol, args.steps, args.warmup, barrier,
                                                  ClockSampler(dev.index))
    ms_max, total_units = aggregate(ms, units * args.steps, dev)
    value = total_units / (ms_max / 1e3) / 1e9
    nnz = [count_nnz(W["theta"], W["z"], W["pitch"], n >> lv, W["nu"] >> lv, W["nu"] >> lv) for lv in range(L)]
    kernels = kernel_table(W, nnz, trace, args.steps)
    roofs = family_rooflines(W, nnz, trace0, peaks, sm_clock, fp32_peak, mp)
    dom = max(roofs, key=lambda k: roofs[k]["avg_launch_ms"] * roofs[k]["launches_timed"]) if roofs else None
    roof = roofs[dom] if dom else {"bound": "onchip-gather", "achieved": None, "peak": None, "unit": "GB/s",
                                   "frac": None, "traffic": None}

    # ---- end to end through the public API with host buffers: every step
    # copies the data b from pinned host memory and the estimate back
    e2e = None
    if not args.no_e2e:
        hb = torch.empty(b.shape, dtype=torch.float32, pin_memory=True)
        hb.copy_(b)
        hv = torch.empty((n, n, n), dtype=torch.float32, pin_memory=True)
        stream = torch.cuda.current_stream()
        bdev = b  # the device buffer the data land in (overwritten every step)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            bdev.copy_(hb, non_blocking=True)
            rec.prepare(bdev)
            rec.iterate(vol)
            hv.copy_(vol, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems = max_over_ranks(e0.elapsed_time(e1))
        e2e = {"value": total_units / (ems / 1e3) / 1e9, "unit": "GUPS", "ms_per_step": ems / args.steps,
               "h2d_bytes_per_step": hb.numel() * 4, "d2h_bytes_per_step": hv.numel() * 4,
               "path": "pinned host b -> device, mgct_multigrid_prepare + mgct_multigrid_iteration, "
                       "estimate -> pinned host, all inside the timed region"}
        del hb, hv

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1 only)
    cpu = None
    sample_vol = None
    if not args.no_cpu and rank == 0 and world == 1:
        import oracle as O
        O.build()
        sample_vol = truth.double().cpu().numpy()
        gups, t, cnt, thr, ta, tat = oracle_sample(args.workload, target_s=args.cpu_seconds, vol=sample_vol)
        cpu = {"value": gups, "unit": "GUPS", "cores": thr, "kind": "oracle",
               "sample": (f"FP64 oracle A and A^T at grid 0 on {cnt} of {K} views ({t:.1f} s)" if n < 1024 else
                          f"FP64 oracle at grid 0: A over one of {K} views ({ta:.1f} s, {thr} threads) and its "
                          f"A^T on {ROW_SAMPLE} of {W['nu']} detector rows scaled to the view ({tat:.1f} s; one "
                          f"thread: the oracle caps its private FP64 volumes at 8 GB)"),
               "oracle_seconds": {"A": ta, "AT": tat}}
    main_name = args.workload
    del rec, vol, b, truth, sample_vol
    g.close()
    W = None
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    # ---- secondary: the 256^3 / 720-view workload (and its time to accuracy)
    second = None
    tta = None
    beside = None
    if not args.no_secondary and main_name != "c2":
        W = make_workload("c2")
        W["name"] = "c2"
        g, b, truth = W["geom"], W["b"], W["truth"]
        n2, K2, L2 = W["n"], W["views"], W["levels"]
        rec = mgct.Reconstructor(g)
        rec.prepare(b)
        vol = torch.zeros((n2, n2, n2), device=dev, dtype=torch.float32)
        ms2, _, tr2, tr20, clk2 = time_steps(rec, vol, 5, 3, barrier, ClockSampler(dev.index))
        u2 = units_per_step(n2, K2, L2)
        nnz2 = [count_nnz(W["theta"], W["z"], W["pitch"], n2 >> lv, W["nu"] >> lv, W["nu"] >> lv)
                for lv in range(L2)]
        second = {"config": workload_config("c2"), "value": u2 * 5 / (ms2 / 1e3) / 1e9, "unit": "GUPS",
                  "ms_per_step": ms2 / 5, "steps": 5, "warmup": 3, "clocks": clk2,
                  "kernels": kernel_table(W, nnz2, tr2, 5),
                  "rooflines": family_rooflines(W, nnz2, tr20, peaks, sm_clock, fp32_peak, mp)}
    elif main_name == "c2":
        W = make_workload("c2")
        W["name"] = "c2"
        g, b, truth = W["geom"], W["b"], W["truth"]
        rec = mgct.Reconstructor(g)
        rec.prepare(b)
        vol = torch.zeros((W["n"],) * 3, device=dev, dtype=torch.float32)

    if W is not None and not args.no_tta and rank == 0:
        tta = time_to_accuracy(args, W, rec, g, b, truth, vol)
        rec.prepare(b)
    if W is not None and not args.no_cpu and not args.no_beside and rank == 0 and world == 1:
        # a side measurement: its failure is reported, not fatal to the line
        try:
            vol_np = truth.double().cpu().numpy()
            _, _, cnt, _, ta, tat = oracle_sample("c2", target_s=args.cpu_seconds, vol=vol_np)
            beside = oracle_beside((cnt, ta, tat, vol_np), (g, b), full_c2=args.oracle_full)
        except Exception as ex:  # noqa: BLE001
            beside = {"error": f"{type(ex).__name__}: {ex}"[:300]}
            try:
                torch.cuda.synchronize()
                torch.cuda.empty_cache()
            except Exception:  # noqa: BLE001
                pass
    if W is not None:
        g.close()

    joint_c4 = None
    if not args.no_joint and rank == 0:
        try:
            joint_c4 = joint_estimation_c4()
        except Exception as ex:  # noqa: BLE001
            joint_c4 = {"error": f"{type(ex).__name__}: {ex}"[:300]}
        torch.cuda.empty_cache()

    hbm = None
    if not args.no_hbm and rank == 0:
        hbm = hbm_kernel_rates(peaks.get("hbm_gbs", 6790.0))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(workload_config(main_name), parallelism=f"replicas x{world}"),
                "roofline": roof, "rooflines": roofs, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk, "kernels": kernels,
                "measured_onchip": mp and {"fp32_tflops": mp["fp32_tflops"], "lds_gbs": mp["lds_gbs"],
                                           "how": "mgct_measure_onchip_peaks: independent FMA chains; "
                                                  "conflict-free 16-byte shared loads"},
                "secondary": second, "hbm_kernels": hbm, "time_to_accuracy": tta, "joint_drift_estimation": joint_c4,
                "oracle_beside": beside}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mgct", choices=["mgct", "reference"])
    ap.add_argument("--workload", default="c5", choices=sorted(WORKLOADS))
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 256^3 / 720-view secondary line (and its time to accuracy)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tta", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-views", type=int, default=8)
    ap.add_argument("--no-beside", action="store_true",
                    help="skip the oracle-beside-GPU timings at 64^3, 256^3, 512^3 and 1024^3")
    ap.add_argument("--oracle-full", action="store_true",
                    help="time the oracle's whole two-iteration solve at 256^3 (minutes of CPU)")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-joint", action="store_true", help="skip the joint drift estimation (256^3, 720 views)")
    ap.add_argument("--eval-1024", action="store_true",
                    help="only the learned correction's evaluation at 1024^3 (plain, PSF kernel, learned)")
    ap.add_argument("--no-hbm", action="store_true", help="skip the HBM-bound kernel rates at 512^3")
    ap.add_argument("--no-literal", action="store_true",
                    help="skip the seconds-to-RMSE<=1e-3 runs on inverse-crime data")
    ap.add_argument("--learn-phantoms", type=int, default=96)
    ap.add_argument("--learn-steps", type=int, default=4000)
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        reference_arm(args, rank)
        return
    if args.eval_1024:
        from paper_2103_10329_gb300 import build
        build.build()
        print(json.dumps({"evaluation_1024": evaluation_1024(args)}), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    gpu_arm(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
