"""The allocation-free residual projection (mgct_project_residual_static)
against the ordinary one (mgct_project with b and sumsq), both called
through the C ABI.

The allocation-free entry point exists for callers that may not allocate
device memory themselves (a plug-in whose host pipeline owns all device
buffers, or a process with a fixed device-memory budget); it keeps its
scratch in one static device array of the library.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2103_10329_gb300 import synth
from tests.helpers import TOL_F32, cuda, gpu_geom, scan_desc, summary, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2103_10329_gb300 import build, mgct
    build.build()
    return mgct.lib()


def _static_call(L, g, level, view0, nviews, stride, vol, out, b, ss):
    st = L.mgct_project_residual_static(g.handle, level, view0, nviews, stride, ctypes.c_void_p(vol.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                        ctypes.c_void_p(ss.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def _check_residual(out, ss, ref, ref_ss, b):
    """The static path against mgct_project.  The two may run different
    projector kernels (the static one reads the plain volume and its
    transpose), each within the float32 per-ray tolerance of the oracle on
    A mu, so their residuals b - A mu agree to TOL_F32 of A mu (not of the
    residual, which may cancel) plus one float32 rounding step of the stored
    difference (2^-23 |b|: the two may round b - A mu to neighbouring
    floats), and their squared norms to 2 TOL_F32 sum |r| |A mu|."""
    r, r_ref, bb = to_np(out), to_np(ref), to_np(b)
    a_ref = bb - r_ref
    den = TOL_F32 * np.maximum(np.abs(a_ref), 1e-2 * np.abs(a_ref).max()) + 2.0 ** -23 * np.abs(bb)
    e = np.abs(r - r_ref) / den
    assert e.max() <= 1.0, summary(e)
    bound = 2 * TOL_F32 * float(np.sum(np.abs(r_ref) * np.abs(a_ref))) + 1e-12 * ref_ss.item()
    assert abs(ss.item() - ref_ss.item()) <= bound, (ss.item(), ref_ss.item(), bound)


def test_static_scratch_matches_allocating_path_twice(L):
    from paper_2103_10329_gb300 import mgct
    d = scan_desc(64, 96, 96, 90, 2104, levels=2)
    g = gpu_geom(d)
    cases = [  # (level, view0, nviews, stride, volume seed): two different calls in a row
        (0, 0, 90, 1, 5),
        (1, 3, 11, 8, 6),
    ]
    for level, v0, cnt, stride, seed in cases:
        n, nu, nv, _, _ = g.level(level)
        vol = cuda(synth.random_volume(n, seed))
        b = cuda(np.random.default_rng(seed).random((cnt, nv, nu)) + 0.5)
        ref_ss = torch.zeros(1, dtype=torch.float64, device="cuda")
        ref = mgct.project(g, vol, level=level, views=(v0, cnt, stride), b=b, sumsq=ref_ss)
        out = torch.full((cnt, nv, nu), float("nan"), device="cuda")
        ss = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert _static_call(L, g, level, v0, cnt, stride, vol, out, b, ss) == 0, L.mgct_last_error()
        torch.cuda.synchronize()
        _check_residual(out, ss, ref, ref_ss, b)


def test_static_scratch_rejects_oversized_requests(L):
    d = scan_desc(256, 48, 48, 4, 1, levels=2)
    g = gpu_geom(d)
    vol = torch.zeros((256, 256, 256), device="cuda")
    out = torch.empty((4, 48, 48), device="cuda")
    b = torch.zeros_like(out)
    ss = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _static_call(L, g, 0, 0, 4, 1, vol, out, b, ss) == -2
    assert b"128^3" in L.mgct_last_error()
    # the coarser grid (128^3) fits
    vol1 = torch.ones((128, 128, 128), device="cuda")
    out1 = torch.empty((4, 24, 24), device="cuda")
    assert _static_call(L, g, 1, 0, 4, 1, vol1, out1, torch.zeros_like(out1), ss) == 0
    torch.cuda.synchronize()
    assert L.mgct_project_residual_static_bytes() > 8 * 2 ** 20


def test_static_scratch_calls_allocate_no_device_memory(L):
    """The property callers rely on: once the library is loaded on the device
    (one warm-up call), further calls of any size within the limits change
    neither the device's free memory nor torch's allocator statistics."""
    from paper_2103_10329_gb300 import mgct
    d = scan_desc(64, 96, 96, 90, 2105, levels=2)
    g = gpu_geom(d)
    calls = []
    for level, v0, cnt, stride, seed in [(0, 0, 90, 1, 7), (1, 2, 20, 4, 8), (0, 5, 33, 2, 9)]:
        n, nu, nv, _, _ = g.level(level)
        vol = cuda(synth.random_volume(n, seed))
        b = cuda(np.random.default_rng(seed).random((cnt, nv, nu)) + 0.5)
        out = torch.empty((cnt, nv, nu), device="cuda")
        ss = torch.empty((1,), dtype=torch.float64, device="cuda")
        ref_ss = torch.zeros(1, dtype=torch.float64, device="cuda")
        ref = mgct.project(g, vol, level=level, views=(v0, cnt, stride), b=b, sumsq=ref_ss)
        calls.append((level, v0, cnt, stride, vol, out, b, ss, ref, ref_ss))
    # warm-up: the first call in this context may load the module (and its array)
    c = calls[0]
    assert _static_call(L, g, *c[:8]) == 0, L.mgct_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for _ in range(2):
        for c in calls:
            assert _static_call(L, g, *c[:8]) == 0, L.mgct_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0, (free0, free1)
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
    for level, v0, cnt, stride, vol, out, b, ss, ref, ref_ss in calls:
        _check_residual(out, ss, ref, ref_ss, b)
