"""FP64 CPU oracle of the preconditioned multigrid Landweber reconstruction.

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the CPU-baseline leg of
the benchmark may import this package; the product (the CUDA library and its
Python binding) never does.  It shares no code with the CUDA path: the
geometry, the projector, every filter and every solver step are written here
again, plainly, in float64 (numpy plus the C file `joseph.c` for the ray
loops).

Each function names the passage of the paper it follows.  Where the paper is
silent the choices below are made, and the CUDA path makes the same ones:

* world units: the volume is the cube [-1/2, 1/2]^3, voxel size h = 1/N at
  the finest grid, 2^g/N on grid g; rotation axis z.
* source s_k = (D cos th, D sin th, z_k); flat detector centred at distance L
  from the source along (-cos th, -sin th, 0), axes e_u = (-sin th, cos th, 0)
  and e_v = (0, 0, 1); the source-to-axis and source-to-detector distances
  are both measured from the source, as Sec. 2 does.  Drift
  phi = (ds_u, ds_v, dd_u, dd_v, psi) shifts the source and detector along
  e_u/e_v (in fine pixels) and turns the detector axes by psi about its normal.
* P (=A) and B (=A^T): Joseph's method, see joseph.c.
* p (Eq. 5): the three 3x3 matrices are stacked along the slice axis (z by
  default); zero padding at the volume edges.
* Restrict (Alg. 1): 2x2x2 mean of mu and 2x2 mean of the log data b.
* Prolongate (Alg. 1): cell-centred trilinear, weights 3/4 and 1/4 per axis,
  edges clamped.
* Landweber (Eq. 4): alpha from an exact line search, <r, A d> / |A d|^2.
* OS-EMTR (Eq. 3): M = 8 subsets, subset m = views k with k mod 8 = m,
  PI = A 1, update only where the denominator exceeds 1e-12 of its maximum.
* Multigrid (Alg. 1): grids 0..L-1; at grid g restrict to g+1, recurse while
  g+1 < L-1 else one OS-EMTR pass on grid g+1; prolongate the coarse change;
  one preconditioned Landweber step; soft threshold (lambda, default 0).

Functions with no independent pin say "parity unpinned" in their docstring.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile joseph.c into _build/liboracle.so with gcc (OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "joseph.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c99",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        i = ctypes.c_int
        lib.orc_project.argtypes = [i, i, i, i, dp, dp, dp, dp, dp, dp]
        lib.orc_backproject.argtypes = [i, i, i, i, dp, dp, dp, dp, dp, dp]
        lib.orc_project_rays.argtypes = [i, dp, dp, dp, dp, dp, i, ip, dp]
        lib.orc_weight.argtypes = [i, dp, dp, dp, dp, i, i, i, i, i]
        lib.orc_weight.restype = ctypes.c_double
        lib.orc_backproject_voxels.argtypes = [i, i, i, i, dp, dp, dp, dp, dp, i, ip, i, dp, ip]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_project_grad.argtypes = [i, i, i, i, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def num_threads() -> int:
    return _load().orc_num_threads()


# ----------------------------------------------------------------------------
# Geometry (Sec. 2, Eq. 1: source and detector positions Theta along the
# trajectory; the conventions are listed in the module docstring)
# ----------------------------------------------------------------------------

@dataclass
class Scan:
    n: int                      # finest volume side N
    nu: int                     # finest detector width U (pixels)
    nv: int                     # finest detector height V
    theta: np.ndarray           # [K] source angle, radians
    z: np.ndarray               # [K] source height, world units
    pitch: float                # finest detector pitch, world units
    src_axis_dist: float = 2.0  # D: source to rotation axis
    src_det_dist: float = 4.0   # L: source to detector
    drift: np.ndarray | None = None  # [K, 5] (ds_u, ds_v, dd_u, dd_v [pixels], psi [rad])
    slice_axis: int = 2         # Eq. 5 outer index: 2 = z, 0 = x
    p_kernel: np.ndarray | None = None  # [3][3][3] preconditioner replacing Eq. 5 (correlation), or None
    extra: dict = field(default_factory=dict)

    @property
    def n_views(self) -> int:
        return len(self.theta)


@dataclass
class LevelGeom:
    n: int
    nu: int
    nv: int
    h: float
    src: np.ndarray   # [K,3]
    det: np.ndarray   # [K,3] centre of pixel (0, 0)
    pu: np.ndarray    # [K,3] one pixel step along u
    pv: np.ndarray    # [K,3] one pixel step along v

    @property
    def n_views(self) -> int:
        return self.src.shape[0]

    def subset(self, views) -> "LevelGeom":
        views = np.asarray(views)
        return LevelGeom(self.n, self.nu, self.nv, self.h, np.ascontiguousarray(self.src[views]),
                         np.ascontiguousarray(self.det[views]), np.ascontiguousarray(self.pu[views]),
                         np.ascontiguousarray(self.pv[views]))


def level_geometry(scan: Scan, level: int = 0) -> LevelGeom:
    """Per-view source, detector pixel (0,0) centre and pixel steps on grid
    `level` (volume N/2^g, detector U/2^g x V/2^g at pitch 2^g Delta; the
    views are not restricted, Alg. 1 passes Theta unchanged)."""
    f = 1 << level
    n, nu, nv = scan.n // f, scan.nu // f, scan.nv // f
    pitch = scan.pitch * f
    th = np.asarray(scan.theta, dtype=np.float64)
    c, s = np.cos(th), np.sin(th)
    zero = np.zeros_like(th)
    eu = np.stack([-s, c, zero], axis=1)
    ev = np.stack([zero, zero, np.ones_like(th)], axis=1)
    nrm = np.stack([-c, -s, zero], axis=1)
    base = np.stack([scan.src_axis_dist * c, scan.src_axis_dist * s, np.asarray(scan.z, np.float64)], axis=1)
    src = base.copy()
    dcen = base + scan.src_det_dist * nrm
    if scan.drift is not None:
        d = np.asarray(scan.drift, dtype=np.float64)
        src = src + (d[:, 0:1] * scan.pitch) * eu + (d[:, 1:2] * scan.pitch) * ev
        dcen = dcen + (d[:, 2:3] * scan.pitch) * eu + (d[:, 3:4] * scan.pitch) * ev
        cp, sp = np.cos(d[:, 4:5]), np.sin(d[:, 4:5])
        eu, ev = cp * eu + sp * ev, -sp * eu + cp * ev
    pu = pitch * eu
    pv = pitch * ev
    det = dcen - 0.5 * (nu - 1) * pu - 0.5 * (nv - 1) * pv
    return LevelGeom(n, nu, nv, 1.0 / n, np.ascontiguousarray(src), np.ascontiguousarray(det),
                     np.ascontiguousarray(pu), np.ascontiguousarray(pv))


def pixel_centres(g: LevelGeom, view: int):
    """World coordinates [V][U][3] of the detector pixel centres of one view."""
    ju = np.arange(g.nu, dtype=np.float64)
    jv = np.arange(g.nv, dtype=np.float64)
    return (g.det[view][None, None, :] + ju[None, :, None] * g.pu[view][None, None, :]
            + jv[:, None, None] * g.pv[view][None, None, :])


# ----------------------------------------------------------------------------
# P and B (Sec. 2: Eq. 1 defines P; Sec. 2.1 defines B as its adjoint)
# ----------------------------------------------------------------------------

def project(g: LevelGeom, vol: np.ndarray) -> np.ndarray:
    """Sinogram [K][V][U] of line integrals P mu (Joseph, see joseph.c)."""
    vol = np.ascontiguousarray(vol, dtype=np.float64)
    assert vol.shape == (g.n, g.n, g.n)
    out = np.empty((g.n_views, g.nv, g.nu), dtype=np.float64)
    rc = _load().orc_project(g.n, g.nu, g.nv, g.n_views, _dp(g.src), _dp(g.det), _dp(g.pu),
                             _dp(g.pv), _dp(vol), _dp(out))
    if rc != 0:
        raise ValueError("geometry produced a ray whose major axis is z")
    return out


def backproject(g: LevelGeom, sino: np.ndarray) -> np.ndarray:
    """Volume [N][N][N] = B y = A^T y, by scattering every ray."""
    sino = np.ascontiguousarray(sino, dtype=np.float64)
    assert sino.shape == (g.n_views, g.nv, g.nu)
    out = np.empty((g.n, g.n, g.n), dtype=np.float64)
    rc = _load().orc_backproject(g.n, g.nu, g.nv, g.n_views, _dp(g.src), _dp(g.det), _dp(g.pu),
                                 _dp(g.pv), _dp(sino), _dp(out))
    if rc != 0:
        raise ValueError("geometry produced a ray whose major axis is z (or out of memory)")
    return out


def project_rays(g: LevelGeom, vol: np.ndarray, rays: np.ndarray) -> np.ndarray:
    """(A vol) at rays[i] = (view, v, u)."""
    vol = np.ascontiguousarray(vol, dtype=np.float64)
    rays = np.ascontiguousarray(rays, dtype=np.int32)
    out = np.empty(len(rays), dtype=np.float64)
    rc = _load().orc_project_rays(g.n, _dp(g.src), _dp(g.det), _dp(g.pu), _dp(g.pv), _dp(vol),
                                  len(rays), _ip(rays), _dp(out))
    if rc != 0:
        raise ValueError("z-major ray")
    return out


def backproject_voxels(g: LevelGeom, sino: np.ndarray, vox: np.ndarray, radius: int = 4):
    """(A^T y) at voxels vox[i] = (x, y, z), from the per-entry weight summed
    over a pixel window per view.  Raises if the window was too small."""
    sino = np.ascontiguousarray(sino, dtype=np.float64)
    vox = np.ascontiguousarray(vox, dtype=np.int32)
    out = np.empty(len(vox), dtype=np.float64)
    edge = np.zeros(len(vox), dtype=np.int32)
    _load().orc_backproject_voxels(g.n, g.nu, g.nv, g.n_views, _dp(g.src), _dp(g.det), _dp(g.pu),
                                   _dp(g.pv), _dp(sino), len(vox), _ip(vox), radius, _dp(out),
                                   _ip(edge))
    if edge.any():
        raise ValueError("pixel window too small for some voxels; raise radius")
    return out


def weight(g: LevelGeom, view: int, ju: int, jv: int, ix: int, iy: int, iz: int) -> float:
    """One entry of A, from the definition (independent of the plane loop)."""
    return _load().orc_weight(g.n, _dp(g.src[view]), _dp(g.det[view]), _dp(g.pu[view]),
                              _dp(g.pv[view]), ju, jv, ix, iy, iz)


# ----------------------------------------------------------------------------
# Per-view geometry gradient (Sec. 1: drift estimated jointly with the image)
# ----------------------------------------------------------------------------

def nominal_axes(scan: Scan):
    """Untilted detector axes e_u, e_v [K,3] along which the drift offsets act."""
    th = np.asarray(scan.theta, dtype=np.float64)
    zero = np.zeros_like(th)
    return (np.stack([-np.sin(th), np.cos(th), zero], axis=1),
            np.stack([zero, zero, np.ones_like(th)], axis=1))


def geometry_grad(scan: Scan, vol: np.ndarray, y: np.ndarray, level: int = 0) -> np.ndarray:
    """d/d phi_k of sum_rays y * (P mu)_ray for phi_k = (ds_u, ds_v, dd_u, dd_v,
    psi): the ray end-point derivatives of joseph.c chained through the
    geometry: ds_u, ds_v move the source by pitch e_u, pitch e_v; dd_u, dd_v
    move every pixel the same way; psi turns the pixel offsets (u' e_u' +
    v' e_v') pitch_g about the detector normal, d/dpsi = u' e_v' - v' e_u'.
    Returns [K, 5]."""
    g = level_geometry(scan, level)
    vol = np.ascontiguousarray(vol, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    K = g.n_views
    gs, gp, gpu, gpv = (np.zeros((K, 3)) for _ in range(4))
    rc = _load().orc_project_grad(g.n, g.nu, g.nv, K, _dp(g.src), _dp(g.det), _dp(g.pu), _dp(g.pv), _dp(vol),
                                  _dp(y), _dp(gs), _dp(gp), _dp(gpu), _dp(gpv))
    if rc != 0:
        raise ValueError("z-major ray")
    eu, ev = nominal_axes(scan)
    p0 = scan.pitch
    out = np.zeros((K, 5))
    out[:, 0] = p0 * np.sum(gs * eu, axis=1)
    out[:, 1] = p0 * np.sum(gs * ev, axis=1)
    out[:, 2] = p0 * np.sum(gp * eu, axis=1)
    out[:, 3] = p0 * np.sum(gp * ev, axis=1)
    # pu, pv are the tilted pixel steps (pitch_g e_u', pitch_g e_v')
    out[:, 4] = np.sum(gpu * g.pv, axis=1) - np.sum(gpv * g.pu, axis=1)
    return out


# ----------------------------------------------------------------------------
# Closed-form line integrals (pins for P; also the noise-free data model Eq. 1)
# ----------------------------------------------------------------------------

def _rays(g: LevelGeom):
    """Source [K,1,1,3] and unit directions [K,V,U,3] of every ray."""
    ju = np.arange(g.nu, dtype=np.float64)
    jv = np.arange(g.nv, dtype=np.float64)
    p = (g.det[:, None, None, :] + ju[None, None, :, None] * g.pu[:, None, None, :]
         + jv[None, :, None, None] * g.pv[:, None, None, :])
    s = g.src[:, None, None, :]
    w = p - s
    w = w / np.linalg.norm(w, axis=-1, keepdims=True)
    return s, w


def ellipsoid_line_integrals(g: LevelGeom, ph: dict) -> np.ndarray:
    """Exact line integrals of the additive ellipsoid phantom along every ray:
    mu_e times the chord length, from the ray/quadric intersection."""
    s, w = _rays(g)
    out = np.zeros(w.shape[:-1])
    for c, ax, rot, mu in zip(ph["centre"], ph["axes"], ph["rot"], ph["mu"]):
        m = rot @ np.diag(1.0 / ax ** 2) @ rot.T
        d = s - c
        A = np.einsum("...i,ij,...j->...", w, m, w)
        B = np.einsum("...i,ij,...j->...", w, m, d)
        C = np.einsum("...i,ij,...j->...", d, m, d) - 1.0
        disc = B * B - A * C
        chord = np.where(disc > 0, 2.0 * np.sqrt(np.maximum(disc, 0.0)) / A, 0.0)
        out += mu * chord
    return out


def blob_line_integrals(g: LevelGeom, ph: dict) -> np.ndarray:
    """Exact line integrals of Gaussian blobs: amp sigma sqrt(2 pi) exp(-d^2/(2 sigma^2)),
    d the distance from the blob centre to the ray's line."""
    s, w = _rays(g)
    out = np.zeros(w.shape[:-1])
    for c, sg, amp in zip(ph["centre"], ph["sigma"], ph["amp"]):
        d = c - s
        along = np.sum(d * w, axis=-1)
        d2 = np.sum(d * d, axis=-1) - along * along
        out += amp * sg * math.sqrt(2 * math.pi) * np.exp(-d2 / (2 * sg * sg))
    return out


# ----------------------------------------------------------------------------
# Preconditioner p (Eq. 5), soft threshold (Alg. 1)
# ----------------------------------------------------------------------------

EQ5 = np.array([
    [[-1, -1, -1], [-1, 0, -1], [-1, -1, -1]],
    [[-8, -4, -8], [-4, 64, -4], [-8, -4, -8]],
    [[-1, -1, -1], [-1, 0, -1], [-1, -1, -1]],
], dtype=np.float64) / 64.0


def eq5_kernel(slice_axis: int = 2) -> np.ndarray:
    """Eq. 5 as a [dz][dy][dx] array.  The outer index of the printed list
    runs along `slice_axis` (2 = z, the rotation axis; 0 = x)."""
    if slice_axis == 2:
        return EQ5.copy()
    if slice_axis == 0:
        return np.ascontiguousarray(np.transpose(EQ5, (1, 2, 0)))
    if slice_axis == 1:
        return np.ascontiguousarray(np.transpose(EQ5, (1, 0, 2)))
    raise ValueError(slice_axis)


def precondition(x: np.ndarray, slice_axis: int = 2, kernel: np.ndarray | None = None) -> np.ndarray:
    """p * x (Eq. 4 and 5): 27-point correlation out(p) = sum_d k[d] x(p + d),
    d in {-1, 0, 1}^3 indexed [dz][dy][dx], zero outside the volume.  Eq. 5
    is symmetric, so convolution and correlation coincide for it; `kernel`
    (a [3][3][3] array) replaces it."""
    k = eq5_kernel(slice_axis) if kernel is None else np.asarray(kernel, dtype=np.float64).reshape(3, 3, 3)
    n0, n1, n2 = x.shape
    pad = np.zeros((n0 + 2, n1 + 2, n2 + 2))
    pad[1:-1, 1:-1, 1:-1] = x
    out = np.zeros(x.shape)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                if k[dz, dy, dx] != 0.0:
                    out += k[dz, dy, dx] * pad[dz:dz + n0, dy:dy + n1, dx:dx + n2]
    return out


def soft_threshold(x: np.ndarray, lam: float) -> np.ndarray:
    """SoftThreshold of Alg. 1: sign(x) max(|x| - lambda, 0)."""
    return np.sign(x) * np.maximum(np.abs(x) - lam, 0.0)


def bilateral_filter(x: np.ndarray, sigma_s: float, sigma_r: float, radius: int) -> np.ndarray:
    """BilateralFilter of Alg. 1 (its parameters are not given in the paper):
        out(p) = sum_q w(p, q) x(q) / sum_q w(p, q),
        w(p, q) = exp(-|p - q|^2 / (2 sigma_s^2)) exp(-(x(p) - x(q))^2 / (2 sigma_r^2)),
    q over the (2 radius + 1)^3 window around p that lies inside the volume
    (distances in voxels of the grid)."""
    x = np.asarray(x, dtype=np.float64)
    n0, n1, n2 = x.shape
    num = np.zeros_like(x)
    den = np.zeros_like(x)
    for dz in range(-radius, radius + 1):
        for dy in range(-radius, radius + 1):
            for dx in range(-radius, radius + 1):
                ws = np.exp(-(dz * dz + dy * dy + dx * dx) / (2.0 * sigma_s * sigma_s))
                # q = p + (dz, dy, dx): the part of the volume where q is inside
                zs, ze = max(0, -dz), min(n0, n0 - dz)
                ys, ye = max(0, -dy), min(n1, n1 - dy)
                xs, xe = max(0, -dx), min(n2, n2 - dx)
                if zs >= ze or ys >= ye or xs >= xe:
                    continue
                xp = x[zs:ze, ys:ye, xs:xe]
                xq = x[zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx]
                w = ws * np.exp(-((xp - xq) ** 2) / (2.0 * sigma_r * sigma_r))
                num[zs:ze, ys:ye, xs:xe] += w * xq
                den[zs:ze, ys:ye, xs:xe] += w
    return num / den


# ----------------------------------------------------------------------------
# Grid transfer (Alg. 1 Restrict / Prolongate)
# ----------------------------------------------------------------------------

def restrict_volume(v: np.ndarray) -> np.ndarray:
    """2x2x2 mean: the attenuation coefficient is intensive."""
    n = v.shape[0] // 2
    return v.reshape(n, 2, n, 2, n, 2).mean(axis=(1, 3, 5))


def restrict_sino(b: np.ndarray) -> np.ndarray:
    """2x2 mean of each view's log data (views unchanged)."""
    k, nv, nu = b.shape
    return b.reshape(k, nv // 2, 2, nu // 2, 2).mean(axis=(2, 4))


def _prolong_axis(c: np.ndarray, axis: int) -> np.ndarray:
    c = np.moveaxis(c, axis, 0)
    m = c.shape[0]
    lo = np.concatenate([c[:1], c[:-1]], axis=0)   # c_{i-1}, clamped
    hi = np.concatenate([c[1:], c[-1:]], axis=0)   # c_{i+1}, clamped
    out = np.empty((2 * m,) + c.shape[1:])
    out[0::2] = 0.75 * c + 0.25 * lo
    out[1::2] = 0.75 * c + 0.25 * hi
    return np.moveaxis(out, 0, axis)


def prolong(c: np.ndarray) -> np.ndarray:
    """Cell-centred trilinear interpolation to the grid twice as fine."""
    out = c
    for ax in range(3):
        out = _prolong_axis(out, ax)
    return out


# ----------------------------------------------------------------------------
# Solvers: Landweber / SIRT (Eq. 2, Eq. 4), OS-EMTR (Eq. 3), multigrid (Alg. 1)
# ----------------------------------------------------------------------------

def landweber_step(g: LevelGeom, mu: np.ndarray, b: np.ndarray, alpha: float | None = None,
                   lam: float = 0.0, precond: bool = True, slice_axis: int = 2,
                   kernel: np.ndarray | None = None):
    """One preconditioned Landweber step (Eq. 4; Eq. 2 when precond=False):
    mu <- S_lambda(mu + alpha p * B(b - P mu)).  alpha=None takes the exact
    line search alpha = <r, A d> / |A d|^2 (0 when A d = 0).
    Returns (mu_new, stats)."""
    r = b - project(g, mu)
    grad = backproject(g, r)
    d = precondition(grad, slice_axis, kernel) if precond else grad
    ad = None
    if alpha is None:
        ad = project(g, d)
        den = float(np.sum(ad * ad))
        alpha = float(np.sum(r * ad)) / den if den > 0 else 0.0
    out = soft_threshold(mu + alpha * d, lam) if lam > 0 else mu + alpha * d
    stats = {"alpha": alpha, "r2": float(np.sum(r * r))}
    if ad is not None:
        stats["r2_pred"] = float(np.sum((r - alpha * ad) ** 2))
    return out, stats


def osemtr_pass(g: LevelGeom, mu: np.ndarray, b: np.ndarray, n_subsets: int = 8,
                pi_sino: np.ndarray | None = None) -> np.ndarray:
    """One full pass of OS-EMTR (Eq. 3) over M = n_subsets ordered subsets
    (subset m = views k with k mod M = m, m = 0..M-1 in order):
        mu <- mu + B{exp(-P mu) - I/I0} / B{exp(-P mu) PI},
    with I/I0 = exp(-b) and PI = P 1 (support = the whole volume); voxels whose
    denominator is not above 1e-12 of its maximum are left unchanged."""
    if pi_sino is None:
        pi_sino = project(g, np.ones((g.n, g.n, g.n)))
    mu = mu.copy()
    for m in range(n_subsets):
        views = np.arange(m, g.n_views, n_subsets)
        if len(views) == 0:
            continue
        gs = g.subset(views)
        t = np.exp(-project(gs, mu))
        num = backproject(gs, t - np.exp(-b[views]))
        den = backproject(gs, t * pi_sino[views])
        dmax = float(den.max())
        mask = den > 1e-12 * dmax if dmax > 0 else np.zeros_like(den, dtype=bool)
        mu[mask] += num[mask] / den[mask]
    return mu


def data_levels(b: np.ndarray, levels: int):
    """b on grids 0..L-1 (Alg. 1 Restrict of the radiographs)."""
    out = [np.asarray(b, dtype=np.float64)]
    for _ in range(1, levels):
        out.append(restrict_sino(out[-1]))
    return out


def multigrid(scan: Scan, mu: np.ndarray, b_levels, levels: int, level: int = 0,
              lam: float = 0.0, n_subsets: int = 8, alpha: float | None = None,
              precond: bool = True, stats: list | None = None, fas: bool = False,
              b: np.ndarray | None = None, bilateral: tuple | None = None) -> np.ndarray:
    """Alg. 1 on grid `level`; returns the updated estimate on that grid.

    The coarse problem's data is the restricted radiographs R b (Alg. 1).
    With fas=True it is instead the full-approximation-scheme data
        b_c = R (b_g - P_g mu) + P_c (R mu),
    b_g being this grid's own data (`b`, else b_levels[level]): a variant
    that is not in the paper (Brandt's FAS coarse equation), under which an
    exact solution of the fine problem is a fixed point of the iteration.
    The plain recursion has no closed form; it is pinned at 8^3 with two and
    three grids against the same reading of Alg. 1 written out with dense
    operators (A from the per-entry weights), and checked against the paper's
    qualitative claim; the FAS form is pinned by its fixed point.  bilateral = (sigma_s, sigma_r, radius)
    applies Alg. 1's BilateralFilter after each grid's Landweber step and soft
    threshold (None: not applied)."""
    g = level_geometry(scan, level)
    mu = np.asarray(mu, dtype=np.float64)
    b_here = b_levels[level] if b is None else np.asarray(b, dtype=np.float64)
    if level + 1 < levels:
        mu_c = restrict_volume(mu)
        if fas:
            b_c = restrict_sino(b_here - project(g, mu)) + project(level_geometry(scan, level + 1), mu_c)
        else:
            b_c = b_levels[level + 1]
        if level + 1 < levels - 1:
            mu_c_new = multigrid(scan, mu_c, b_levels, levels, level + 1, lam, n_subsets,
                                 alpha, precond, stats, fas=fas, b=b_c, bilateral=bilateral)
        else:
            mu_c_new = osemtr_pass(level_geometry(scan, level + 1), mu_c, b_c, n_subsets)
        mu = mu + prolong(mu_c_new - mu_c)
    mu, st = landweber_step(g, mu, b_here, alpha=alpha, lam=lam, precond=precond,
                            slice_axis=scan.slice_axis, kernel=scan.p_kernel)
    if bilateral is not None:
        mu = bilateral_filter(mu, *bilateral)
    if stats is not None:
        st["level"] = level
        stats.append(st)
    return mu


def reconstruct(scan: Scan, b: np.ndarray, iters: int = 2, levels: int = 2, lam: float = 0.0,
                n_subsets: int = 8, mu0: np.ndarray | None = None, stats: list | None = None,
                fas: bool = False, bilateral: tuple | None = None):
    """`iters` multigrid iterations at grid 0 from mu = 0 (Fig. 3: one or two);
    fas=True takes the FAS coarse data (see multigrid)."""
    bl = data_levels(b, levels)
    mu = np.zeros((scan.n,) * 3) if mu0 is None else np.asarray(mu0, dtype=np.float64)
    for _ in range(iters):
        mu = multigrid(scan, mu, bl, levels, 0, lam, n_subsets, stats=stats, fas=fas, bilateral=bilateral)
    return mu


def sirt(scan: Scan, b: np.ndarray, iters: int, alpha: float | None = None):
    """Plain Landweber / SIRT (Eq. 2) on grid 0, line-searched step."""
    g = level_geometry(scan, 0)
    mu = np.zeros((scan.n,) * 3)
    for _ in range(iters):
        mu, _ = landweber_step(g, mu, b, alpha=alpha, precond=False)
    return mu
