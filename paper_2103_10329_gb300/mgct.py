"""Thin Python binding of libmgct.so (include/mgct.h): argument marshalling
only.  Every operation runs in the library's CUDA kernels; torch supplies the
device memory and the current stream.  There is no CPU fallback: if the
library is missing or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmgct.so")

F32, BF16, F16 = 0, 1, 2
WS_LANDWEBER, WS_OSEMTR, WS_MULTIGRID = 0, 1, 2
_DT = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}
_TD = {v: k for k, v in _DT.items()}


class MgctError(RuntimeError):
    pass


class GeomDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nu", ctypes.c_int32), ("nv", ctypes.c_int32),
                ("n_views", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("src_axis_dist", ctypes.c_double), ("src_det_dist", ctypes.c_double),
                ("pixel_pitch", ctypes.c_double),
                ("theta", ctypes.POINTER(ctypes.c_double)), ("z", ctypes.POINTER(ctypes.c_double)),
                ("drift", ctypes.POINTER(ctypes.c_double)), ("p_slice_axis", ctypes.c_int32)]


class LwOpts(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("precondition", ctypes.c_int32), ("n_subsets", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("coarse_fas", ctypes.c_int32),
                ("learned_corr", ctypes.c_void_p),
                ("bilateral_sigma_s", ctypes.c_double), ("bilateral_sigma_r", ctypes.c_double),
                ("bilateral_radius", ctypes.c_int32), ("reserved1", ctypes.c_int32)]


_lib = None


def lib():
    """Load the in-tree library (built by paper_2103_10329_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise MgctError(f"{LIB_PATH} is missing: run paper_2103_10329_gb300.build.build() first")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    L.mgct_geometry_create.argtypes = [ctypes.POINTER(GeomDesc), ctypes.POINTER(vp)]
    L.mgct_geometry_set_drift.argtypes = [vp, vp]
    L.mgct_geometry_set_preconditioner.argtypes = [vp, vp]
    L.mgct_bilateral.argtypes = [i, vp, vp, d, d, i, vp]
    L.mgct_check_bounded_wait.argtypes = [d, vp, vp]
    L.mgct_measure_onchip_peaks.argtypes = [vp, vp, vp]
    for fn in ("mgct_geometry_set_preconditioner", "mgct_bilateral", "mgct_check_bounded_wait",
               "mgct_measure_onchip_peaks"):
        getattr(L, fn).restype = ctypes.c_int
    L.mgct_geometry_destroy.argtypes = [vp]
    L.mgct_geometry_destroy.restype = None
    L.mgct_geometry_level.argtypes = [vp, i, vp, vp, vp, vp, vp]
    L.mgct_project.argtypes = [vp, i, i, i, i, vp, i, vp, i, vp, vp, vp]
    L.mgct_backproject.argtypes = [vp, i, i, i, i, vp, i, vp, i, vp]
    L.mgct_precondition.argtypes = [vp, i, vp, vp, vp]
    L.mgct_restrict_volume.argtypes = [i, vp, vp, vp]
    L.mgct_restrict_sino.argtypes = [i, i, i, vp, vp, vp]
    L.mgct_prolong_add.argtypes = [i, vp, vp, vp, vp]
    L.mgct_workspace_bytes.argtypes = [vp, i, i]
    L.mgct_workspace_bytes.restype = sz
    L.mgct_landweber_step.argtypes = [vp, i, vp, vp, vp, sz, ctypes.POINTER(LwOpts), vp, vp]
    L.mgct_osemtr_pass.argtypes = [vp, i, i, vp, vp, vp, vp, sz, vp]
    L.mgct_multigrid_prepare.argtypes = [vp, vp, vp, sz, vp]
    L.mgct_multigrid_iteration.argtypes = [vp, vp, vp, vp, sz, ctypes.POINTER(LwOpts), vp, vp]
    L.mgct_status_string.argtypes = [i]
    L.mgct_status_string.restype = ctypes.c_char_p
    L.mgct_last_error.restype = ctypes.c_char_p
    L.mgct_launch_count.argtypes = [i]
    L.mgct_launch_count.restype = ctypes.c_uint64
    L.mgct_trace_enable.argtypes = [i]
    L.mgct_trace_read.argtypes = [vp, vp, i]
    L.mgct_trace_read_level.argtypes = [i, vp, vp, i]
    L.mgct_multigrid_coarse.argtypes = [vp, vp, vp, vp, sz, ctypes.POINTER(LwOpts), vp, vp]
    L.mgct_landweber_direction.argtypes = [vp, i, vp, vp, vp, sz, ctypes.POINTER(LwOpts), vp, vp, vp]
    L.mgct_landweber_learned.argtypes = [vp, i, vp, vp, vp, sz, ctypes.POINTER(LwOpts), vp, vp, sz, vp, vp]
    L.mgct_axpy.argtypes = [sz, ctypes.c_float, vp, vp, vp]
    for fn in ("mgct_multigrid_coarse", "mgct_landweber_direction", "mgct_landweber_learned", "mgct_axpy"):
        getattr(L, fn).restype = ctypes.c_int
    L.mgct_geometry_grad.argtypes = [vp, i, i, i, i, vp, vp, vp, vp]
    L.mgct_geometry_grad.restype = ctypes.c_int
    L.mgct_project_residual_static.argtypes = [vp, i, i, i, i, vp, vp, vp, vp, vp]
    L.mgct_project_residual_static.restype = ctypes.c_int
    L.mgct_project_residual_static_bytes.restype = sz
    for fn in ("mgct_geometry_create", "mgct_geometry_set_drift", "mgct_geometry_level", "mgct_project",
               "mgct_backproject", "mgct_precondition", "mgct_restrict_volume", "mgct_restrict_sino",
               "mgct_prolong_add", "mgct_landweber_step", "mgct_osemtr_pass", "mgct_multigrid_prepare",
               "mgct_multigrid_iteration"):
        getattr(L, fn).restype = ctypes.c_int
    _lib = L
    return L


def _check(st: int):
    if st != 0:
        L = lib()
        raise MgctError(f"{L.mgct_status_string(st).decode()} ({st}): {L.mgct_last_error().decode()}")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor | None, name: str, dtype=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise MgctError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise MgctError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise MgctError(f"{name} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def launch_count(reset: bool = False) -> int:
    return int(lib().mgct_launch_count(1 if reset else 0))


def check_bounded_wait(seconds: float = 0.2) -> bool:
    """Run the library's bounded device wait on a barrier nothing completes
    (mgct_check_bounded_wait); True when it expired and reported as designed."""
    L = lib()
    flag = ctypes.c_int(0)
    _check(L.mgct_check_bounded_wait(float(seconds), ctypes.byref(flag), _stream()))
    return flag.value == 1


def measure_onchip_peaks() -> dict:
    """The FP32 FMA rate (TFLOP/s) and the shared-memory load bandwidth (GB/s)
    of the current device, measured by the library (mgct_measure_onchip_peaks)."""
    L = lib()
    fp32, lds = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(L.mgct_measure_onchip_peaks(ctypes.byref(fp32), ctypes.byref(lds), _stream()))
    return {"fp32_tflops": fp32.value, "lds_gbs": lds.value}


TRACE_KINDS = ("project", "backproject", "precondition", "transpose", "grid", "update", "reduce",
               "geomgrad", "conv", "other")


def trace_enable(on: bool = True):
    _check(lib().mgct_trace_enable(1 if on else 0))


def trace_read(level: int | None = None) -> dict:
    """{kind: (milliseconds, launches)} of the kernels traced since enable
    (only those made for grid `level` when given)."""
    ms = (ctypes.c_double * len(TRACE_KINDS))()
    cnt = (ctypes.c_uint64 * len(TRACE_KINDS))()
    if level is None:
        _check(lib().mgct_trace_read(ms, cnt, len(TRACE_KINDS)))
    else:
        _check(lib().mgct_trace_read_level(int(level), ms, cnt, len(TRACE_KINDS)))
    return {k: (ms[i], int(cnt[i])) for i, k in enumerate(TRACE_KINDS)}


class Geometry:
    """Owns an mgct_geom handle (mgct_geometry_create)."""

    def __init__(self, n, nu, nv, theta, z, pitch, levels=1, src_axis_dist=2.0, src_det_dist=4.0,
                 drift=None, p_slice_axis=2):
        L = lib()
        self.theta = np.ascontiguousarray(theta, dtype=np.float64)
        self.z = np.ascontiguousarray(z, dtype=np.float64)
        self.n, self.nu, self.nv, self.levels = int(n), int(nu), int(nv), int(levels)
        self.n_views = len(self.theta)
        self.pitch = float(pitch)
        self.src_axis_dist, self.src_det_dist = float(src_axis_dist), float(src_det_dist)
        self.p_slice_axis = int(p_slice_axis)
        self._drift = None if drift is None else np.ascontiguousarray(drift, dtype=np.float64).reshape(-1)
        dp = ctypes.POINTER(ctypes.c_double)
        desc = GeomDesc(self.n, self.nu, self.nv, self.n_views, self.levels, self.src_axis_dist,
                        self.src_det_dist, self.pitch, self.theta.ctypes.data_as(dp),
                        self.z.ctypes.data_as(dp),
                        self._drift.ctypes.data_as(dp) if self._drift is not None else None,
                        self.p_slice_axis)
        h = ctypes.c_void_p()
        _check(L.mgct_geometry_create(ctypes.byref(desc), ctypes.byref(h)))
        self.handle = h

    def set_drift(self, drift):
        self._drift = None if drift is None else np.ascontiguousarray(drift, dtype=np.float64).reshape(-1)
        _check(lib().mgct_geometry_set_drift(
            self.handle, None if self._drift is None else ctypes.c_void_p(self._drift.ctypes.data)))

    def set_preconditioner(self, kernel=None):
        """A [3][3][3] kernel ([dz][dy][dx], applied as a correlation) in place
        of Eq. 5 on every grid; None restores Eq. 5."""
        L = lib()
        if kernel is None:
            _check(L.mgct_geometry_set_preconditioner(self.handle, None))
            return
        k = np.ascontiguousarray(kernel, dtype=np.float64).reshape(27)
        _check(L.mgct_geometry_set_preconditioner(self.handle, ctypes.c_void_p(k.ctypes.data)))

    def level(self, g: int):
        n, nu, nv = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        h, p = ctypes.c_double(), ctypes.c_double()
        _check(lib().mgct_geometry_level(self.handle, g, ctypes.byref(n), ctypes.byref(nu), ctypes.byref(nv),
                                         ctypes.byref(h), ctypes.byref(p)))
        return n.value, nu.value, nv.value, h.value, p.value

    def workspace_bytes(self, op: int, level: int = 0) -> int:
        return int(lib().mgct_workspace_bytes(self.handle, op, level))

    def close(self):
        if getattr(self, "handle", None):
            lib().mgct_geometry_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def geometry_create(*args, **kw) -> Geometry:
    return Geometry(*args, **kw)


def _views(geom: Geometry, views):
    if views is None:
        return 0, geom.n_views, 1
    v0, cnt, stride = views
    return int(v0), int(cnt), int(stride)


def project(geom: Geometry, vol: torch.Tensor, level: int = 0, views=None, out=None,
            out_dtype=torch.float32, b: torch.Tensor | None = None, sumsq: torch.Tensor | None = None):
    """A vol (or b - A vol) for views (view0, count, stride); returns out."""
    v0, cnt, stride = _views(geom, views)
    n, nu, nv, _, _ = geom.level(level)
    if vol.shape != (n, n, n):
        raise MgctError(f"vol must be [{n}]^3, got {tuple(vol.shape)}")
    if out is None:
        out = torch.empty((cnt, nv, nu), device=vol.device, dtype=out_dtype)
    if out.shape != (cnt, nv, nu):
        raise MgctError("out has the wrong shape")
    if b is not None and b.shape != out.shape:
        raise MgctError("b must match out")
    _check(lib().mgct_project(geom.handle, level, v0, cnt, stride, _ptr(vol, "vol"), _DT[vol.dtype],
                              _ptr(out, "out"), _DT[out.dtype], _ptr(b, "b", torch.float32),
                              _ptr(sumsq, "sumsq", torch.float64), _stream()))
    return out


def backproject(geom: Geometry, sino: torch.Tensor, level: int = 0, views=None, out=None,
                accumulate: bool = False):
    """A^T sino (float32 volume)."""
    v0, cnt, stride = _views(geom, views)
    n, nu, nv, _, _ = geom.level(level)
    if sino.shape != (cnt, nv, nu):
        raise MgctError(f"sino must be [{cnt}][{nv}][{nu}], got {tuple(sino.shape)}")
    if out is None:
        out = torch.empty((n, n, n), device=sino.device, dtype=torch.float32)
    _check(lib().mgct_backproject(geom.handle, level, v0, cnt, stride, _ptr(sino, "sino"), _DT[sino.dtype],
                                  _ptr(out, "out", torch.float32), 1 if accumulate else 0, _stream()))
    return out


def geometry_grad(geom: Geometry, vol: torch.Tensor, y: torch.Tensor, level: int = 0, views=None, out=None):
    """d/dphi of sum y * (A vol) per view, phi = (ds_u, ds_v, dd_u, dd_v, psi): float64 [nviews, 5]."""
    v0, cnt, stride = _views(geom, views)
    if out is None:
        out = torch.empty((cnt, 5), device=vol.device, dtype=torch.float64)
    _check(lib().mgct_geometry_grad(geom.handle, level, v0, cnt, stride, _ptr(vol, "vol", torch.float32),
                                    _ptr(y, "y", torch.float32), _ptr(out, "out", torch.float64), _stream()))
    return out


def precondition(geom: Geometry, x: torch.Tensor, level: int = 0, out=None):
    """p * x (Eq. 5)."""
    if out is None:
        out = torch.empty_like(x)
    _check(lib().mgct_precondition(geom.handle, level, _ptr(x, "x", torch.float32),
                                   _ptr(out, "out", torch.float32), _stream()))
    return out


def restrict_volume(x: torch.Tensor, out=None):
    n = x.shape[0]
    if out is None:
        out = torch.empty((n // 2,) * 3, device=x.device, dtype=torch.float32)
    _check(lib().mgct_restrict_volume(n, _ptr(x, "x", torch.float32), _ptr(out, "out", torch.float32), _stream()))
    return out


def restrict_sino(b: torch.Tensor, out=None):
    k, nv, nu = b.shape
    if out is None:
        out = torch.empty((k, nv // 2, nu // 2), device=b.device, dtype=torch.float32)
    _check(lib().mgct_restrict_sino(k, nv, nu, _ptr(b, "b", torch.float32), _ptr(out, "out", torch.float32),
                                    _stream()))
    return out


def prolong_add(coarse_new: torch.Tensor, coarse_old: torch.Tensor, fine: torch.Tensor):
    _check(lib().mgct_prolong_add(coarse_new.shape[0], _ptr(coarse_new, "coarse_new", torch.float32),
                                  _ptr(coarse_old, "coarse_old", torch.float32),
                                  _ptr(fine, "fine", torch.float32), _stream()))
    return fine


def workspace(geom: Geometry, op: int, level: int = 0, device="cuda") -> torch.Tensor:
    nbytes = geom.workspace_bytes(op, level)
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def _opts(alpha, lam, precond, n_subsets, storage=torch.float32, fas=False, bilateral=None):
    ss, sr, r = bilateral if bilateral is not None else (0.0, 0.0, 0)
    return LwOpts(float(alpha) if alpha is not None else 0.0, float(lam), 1 if precond else 0,
                  int(n_subsets), _DT[storage], 1 if fas else 0, None, float(ss), float(sr), int(r), 0)


def landweber_step(geom: Geometry, vol: torch.Tensor, b: torch.Tensor, level: int = 0, alpha=None,
                   lam: float = 0.0, precond: bool = True, ws: torch.Tensor | None = None,
                   stats: torch.Tensor | None = None, storage=torch.float32):
    """One (preconditioned) Landweber step in place; stats: float64[4] device
    tensor (alpha, r2, r2_pred, nonfinite) or None; storage: dtype of the
    copies the projector and back-projector read (float32, bfloat16, float16)."""
    if ws is None:
        ws = workspace(geom, WS_LANDWEBER, level, vol.device)
    o = _opts(alpha, lam, precond, 0, storage)
    _check(lib().mgct_landweber_step(geom.handle, level, _ptr(vol, "vol", torch.float32),
                                     _ptr(b, "b", torch.float32), _ptr(ws, "ws"), ws.numel(), ctypes.byref(o),
                                     _ptr(stats, "stats", torch.float64), _stream()))
    return vol


def osemtr_pass(geom: Geometry, vol: torch.Tensor, b: torch.Tensor, pi: torch.Tensor, level: int = 0,
                n_subsets: int = 8, ws: torch.Tensor | None = None):
    if ws is None:
        ws = workspace(geom, WS_OSEMTR, level, vol.device)
    _check(lib().mgct_osemtr_pass(geom.handle, level, n_subsets, _ptr(vol, "vol", torch.float32),
                                  _ptr(b, "b", torch.float32), _ptr(pi, "pi", torch.float32), _ptr(ws, "ws"),
                                  ws.numel(), _stream()))
    return vol


def multigrid_prepare(geom: Geometry, b: torch.Tensor, ws: torch.Tensor):
    _check(lib().mgct_multigrid_prepare(geom.handle, _ptr(b, "b", torch.float32), _ptr(ws, "ws"), ws.numel(),
                                        _stream()))


def multigrid_iteration(geom: Geometry, vol: torch.Tensor, b: torch.Tensor, ws: torch.Tensor, alpha=None,
                        lam: float = 0.0, precond: bool = True, n_subsets: int = 8,
                        stats: torch.Tensor | None = None, storage=torch.float32, fas: bool = False,
                        bilateral=None):
    """One Alg. 1 iteration at grid 0; fas=True takes the full-approximation-
    scheme coarse data R(b - A mu) + A_c(R mu) (a variant outside the paper);
    bilateral = (sigma_s, sigma_r, radius) applies Alg. 1's BilateralFilter
    after each grid's Landweber step."""
    o = _opts(alpha, lam, precond, n_subsets, storage, fas, bilateral)
    _check(lib().mgct_multigrid_iteration(geom.handle, _ptr(vol, "vol", torch.float32),
                                          _ptr(b, "b", torch.float32), _ptr(ws, "ws"), ws.numel(),
                                          ctypes.byref(o), _ptr(stats, "stats", torch.float64), _stream()))
    return vol


def multigrid_coarse(geom: Geometry, vol: torch.Tensor, ws: torch.Tensor, n_subsets: int = 8,
                     stats: torch.Tensor | None = None, storage=torch.float32, lam: float = 0.0,
                     b: torch.Tensor | None = None, fas: bool = False, bilateral=None):
    """Alg. 1 without the grid-0 Landweber step; b (grid-0 data) is needed
    with fas=True."""
    o = _opts(None, lam, True, n_subsets, storage, fas, bilateral)
    _check(lib().mgct_multigrid_coarse(geom.handle, _ptr(vol, "vol", torch.float32), _ptr(b, "b", torch.float32),
                                       _ptr(ws, "ws"), ws.numel(), ctypes.byref(o),
                                       _ptr(stats, "stats", torch.float64), _stream()))
    return vol


def landweber_direction(geom: Geometry, vol: torch.Tensor, b: torch.Tensor, level: int = 0,
                        ws: torch.Tensor | None = None, out: torch.Tensor | None = None, precond: bool = True,
                        stats: torch.Tensor | None = None, storage=torch.float32):
    """The step alpha d of one Landweber step, without updating vol."""
    if ws is None:
        ws = workspace(geom, WS_LANDWEBER, level, vol.device)
    if out is None:
        out = torch.empty_like(vol)
    o = _opts(None, 0.0, precond, 0, storage)
    _check(lib().mgct_landweber_direction(geom.handle, level, _ptr(vol, "vol", torch.float32),
                                          _ptr(b, "b", torch.float32), _ptr(ws, "ws"), ws.numel(), ctypes.byref(o),
                                          _ptr(out, "out", torch.float32), _ptr(stats, "stats", torch.float64),
                                          _stream()))
    return out


def landweber_learned(geom: Geometry, vol: torch.Tensor, b: torch.Tensor, net: "Net", level: int = 0,
                      ws: torch.Tensor | None = None, stats: torch.Tensor | None = None, storage=torch.float32,
                      lam: float = 0.0):
    """Learned Landweber step in place (mgct_landweber_learned); stats float64[8]."""
    if ws is None:
        ws = workspace(geom, WS_LANDWEBER, level, vol.device)
    if stats is None:
        stats = torch.zeros(8, dtype=torch.float64, device=vol.device)
    nws = net._workspace(vol.numel(), False, plane=int(vol.shape[-1] * vol.shape[-2]))
    o = _opts(None, lam, True, 0, storage)
    _check(lib().mgct_landweber_learned(geom.handle, level, _ptr(vol, "vol", torch.float32),
                                        _ptr(b, "b", torch.float32), _ptr(ws, "ws"), ws.numel(), ctypes.byref(o),
                                        net.handle, _ptr(nws, "net_ws"), nws.numel(),
                                        _ptr(stats, "stats", torch.float64), _stream()))
    return vol


def bilateral(x: torch.Tensor, sigma_s: float, sigma_r: float, radius: int, out: torch.Tensor | None = None):
    """Alg. 1 BilateralFilter of a float32 [n]^3 volume (mgct_bilateral)."""
    n = x.shape[0]
    if out is None:
        out = torch.empty_like(x)
    L = lib()
    _check(L.mgct_bilateral(n, _ptr(x, "x", torch.float32), _ptr(out, "out", torch.float32), float(sigma_s),
                            float(sigma_r), int(radius), _stream()))
    return out


def axpy(a: float, x: torch.Tensor, y: torch.Tensor):
    """y += a x (float32)."""
    _check(lib().mgct_axpy(x.numel(), ctypes.c_float(a), _ptr(x, "x", torch.float32), _ptr(y, "y", torch.float32),
                           _stream()))
    return y


class Reconstructor:
    """Alg. 1 driver state: a geometry with `levels` grids and its multigrid
    workspace.  `prepare(b)` once per data set, then `iterate(vol)`."""

    def __init__(self, geom: Geometry, device="cuda"):
        self.geom = geom
        self.ws = workspace(geom, WS_MULTIGRID, 0, device)
        self.stats = torch.zeros((max(geom.levels, 1), 4), dtype=torch.float64, device=device)
        self.b = None

    def prepare(self, b: torch.Tensor):
        self.b = b
        multigrid_prepare(self.geom, b, self.ws)

    def iterate(self, vol: torch.Tensor, **kw):
        return multigrid_iteration(self.geom, vol, self.b, self.ws, stats=self.stats, **kw)

    def reconstruct(self, iters: int = 2, **kw):
        n = self.geom.n
        vol = torch.zeros((n, n, n), device=self.ws.device, dtype=torch.float32)
        for _ in range(iters):
            self.iterate(vol, **kw)
        return vol

    def iterate_learned(self, vol: torch.Tensor, net: "Net", storage=torch.float32, n_subsets: int = 8,
                        fas: bool = False):
        """Alg. 1 with the learned Landweber step on grid 0 (coarse grids plain)."""
        if self.geom.levels > 1:
            multigrid_coarse(self.geom, vol, self.ws, n_subsets=n_subsets, stats=self.stats, storage=storage,
                             b=self.b, fas=fas)
        if not hasattr(self, "_lw_ws"):
            self._lw_ws = workspace(self.geom, WS_LANDWEBER, 0, vol.device)
            self.learned_stats = torch.zeros(8, dtype=torch.float64, device=vol.device)
        return landweber_learned(self.geom, vol, self.b, net, ws=self._lw_ws, stats=self.learned_stats,
                                 storage=storage)


def project_residual_static(geom: Geometry, vol: torch.Tensor, b: torch.Tensor, sumsq: torch.Tensor,
                            level: int = 0, views=None, out=None):
    """out = b - A vol and sumsq[0] = |out|^2, computed with the library's
    static scratch instead of any allocation (mgct_project_residual_static):
    for callers that may not allocate device memory themselves.  Volumes up
    to 128^3; overlapping calls on different streams race on the scratch."""
    v0, cnt, stride = _views(geom, views)
    n, nu, nv, _, _ = geom.level(level)
    if out is None:
        out = torch.empty((cnt, nv, nu), device=vol.device, dtype=torch.float32)
    _check(lib().mgct_project_residual_static(geom.handle, level, v0, cnt, stride, _ptr(vol, "vol", torch.float32),
                                              _ptr(out, "out", torch.float32), _ptr(b, "b", torch.float32),
                                              _ptr(sumsq, "sumsq", torch.float64), _stream()))
    return out


# ---------------------------------------------------------------------------
# learned preconditioner correction (mgct_net_*)
# ---------------------------------------------------------------------------
_net_sigs_done = False


def _net_sigs():
    global _net_sigs_done
    if _net_sigs_done:
        return lib()
    L = lib()
    vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    L.mgct_net_create.argtypes = [ctypes.c_uint64, ctypes.POINTER(vp)]
    L.mgct_net_destroy.argtypes = [vp]
    L.mgct_net_destroy.restype = None
    L.mgct_net_param_count.restype = sz
    L.mgct_net_set_params.argtypes = [vp, vp, sz]
    L.mgct_net_get_params.argtypes = [vp, vp, sz]
    L.mgct_net_get_grads.argtypes = [vp, vp, sz]
    L.mgct_net_workspace_bytes.argtypes = [ctypes.c_int64, i]
    L.mgct_net_workspace_bytes.restype = sz
    L.mgct_net_apply.argtypes = [vp, i, i, i, i, vp, vp, vp, sz, vp]
    L.mgct_net_forward_backward.argtypes = [vp, i, i, i, i, vp, vp, vp, sz, vp, vp]
    L.mgct_net_adam_step.argtypes = [vp, ctypes.c_double, vp]
    L.mgct_net_check.argtypes = [vp, vp]
    for fn in ("mgct_net_create", "mgct_net_set_params", "mgct_net_get_params", "mgct_net_get_grads",
               "mgct_net_apply", "mgct_net_forward_backward", "mgct_net_adam_step", "mgct_net_check"):
        getattr(L, fn).restype = ctypes.c_int
    _net_sigs_done = True
    return L


class Net:
    """The learned correction network (mgct_net_create)."""

    def __init__(self, seed: int = 0):
        L = _net_sigs()
        h = ctypes.c_void_p()
        _check(L.mgct_net_create(ctypes.c_uint64(seed), ctypes.byref(h)))
        self.handle = h
        self.count = int(L.mgct_net_param_count())
        self._ws = None
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")

    def params(self) -> np.ndarray:
        out = np.empty(self.count, dtype=np.float32)
        _check(_net_sigs().mgct_net_get_params(self.handle, out.ctypes.data, self.count))
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(_net_sigs().mgct_net_set_params(self.handle, p.ctypes.data, p.size))

    def grads(self) -> np.ndarray:
        out = np.empty(self.count, dtype=np.float32)
        _check(_net_sigs().mgct_net_get_grads(self.handle, out.ctypes.data, self.count))
        return out

    # inference workspaces above this size are replaced by a z-slab workspace
    # (mgct_net_apply then runs the volume slab by slab)
    SLAB_BYTES = 16 << 30

    def _workspace(self, nvox: int, training: bool, plane: int | None = None,
                   slab_planes: int | None = None) -> torch.Tensor:
        L = _net_sigs()
        need = int(L.mgct_net_workspace_bytes(nvox, 1 if training else 0))
        if not training and plane and (slab_planes is not None or need > self.SLAB_BYTES):
            if slab_planes is None:
                per_plane = int(L.mgct_net_workspace_bytes(plane, 0))
                slab_planes = max(1, self.SLAB_BYTES // per_plane - 8)
            need = min(need, int(L.mgct_net_workspace_bytes((slab_planes + 8) * plane, 0)))
        if self._ws is None or self._ws.numel() < need:
            self._ws = None
            self._ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        return self._ws[:need]

    def apply(self, step: torch.Tensor, out: torch.Tensor | None = None,
              slab_planes: int | None = None) -> torch.Tensor:
        """Corrected step s (x + f(x)), x = step / RMS(step); step [B][D][H][W] or [D][H][W].
        Volumes whose workspace would exceed SLAB_BYTES (or any volume, with
        slab_planes) run in z-slabs of that many planes plus a 4-plane halo."""
        shp = step.shape if step.dim() == 4 else (1,) + tuple(step.shape)
        if out is None:
            out = torch.empty_like(step)
        ws = self._workspace(int(np.prod(shp)), False, plane=int(shp[2] * shp[3]), slab_planes=slab_planes)
        _check(_net_sigs().mgct_net_apply(self.handle, *shp, _ptr(step, "step", torch.float32),
                                          _ptr(out, "out", torch.float32), _ptr(ws, "ws"), ws.numel(), _stream()))
        return out

    def forward_backward(self, x: torch.Tensor, t: torch.Tensor) -> torch.Tensor:
        """Loss mean((x + f(x) - t)^2) (device float64) and parameter gradients."""
        shp = x.shape if x.dim() == 4 else (1,) + tuple(x.shape)
        ws = self._workspace(int(np.prod(shp)), True)
        _check(_net_sigs().mgct_net_forward_backward(self.handle, *shp, _ptr(x, "x", torch.float32),
                                                     _ptr(t, "t", torch.float32), _ptr(ws, "ws"), ws.numel(),
                                                     _ptr(self.loss, "loss", torch.float64), _stream()))
        return self.loss

    def adam_step(self, lr: float) -> None:
        _check(_net_sigs().mgct_net_adam_step(self.handle, float(lr), _stream()))

    def check(self) -> None:
        """Synchronise and raise if a convolution's bounded wait expired
        (mgct_net_check)."""
        _check(_net_sigs().mgct_net_check(self.handle, _stream()))

    def close(self):
        if getattr(self, "handle", None):
            _net_sigs().mgct_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
