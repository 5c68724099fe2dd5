"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the bench.

This module holds input generation only: the source trajectory's parameters,
random phantom descriptions (ellipsoids, Gaussian blobs, a porous texture),
their voxelisation, per-view drift random walks and photon noise.  It holds
none of the reconstruction method's arithmetic (no projector, no filter, no
grid transfer, no solver), so sharing it between the oracle and the GPU path
shares data, not code.

World units: the reconstruction volume is the cube [-1/2, 1/2]^3 (width 1,
half-width R = 1/2); voxel i of an N-voxel axis has its centre at
(i - (N-1)/2)/N.  Volumes are returned in [z][y][x] order, x fastest.
"""
from __future__ import annotations

import math

import numpy as np
import torch

R_HALF = 0.5  # half-width of the reconstruction cube, world units


def trajectory(n_views: int, seed: int):
    """Space-filling source trajectory (Sec. 1, Sec. 2: a "complete" trajectory).

    The paper's own trajectory (stride 15.3 degrees, its ref. [4]) is not given
    in the text; this is the golden-ratio stand-in: theta_k = 2*pi*frac(0.618034*k)
    and z_k stratified uniformly over the volume height, one random offset per
    stratum.  Returns float64 arrays (theta [K], z [K]).
    """
    k = np.arange(n_views, dtype=np.float64)
    theta = 2.0 * np.pi * np.mod(0.618034 * k, 1.0)
    rng = np.random.default_rng(seed)
    u = rng.random(n_views)
    z = -R_HALF + 2.0 * R_HALF * (k + u) / n_views
    return theta, z


def drift_walk(n_views: int, seed: int, sigma_px: float = 0.3,
               half_diag_px: float = 1.0):
    """Per-view geometry drift phi_k = (ds_u, ds_v, dd_u, dd_v, psi) as Gaussian
    random walks (the thermal drift the paper motivates in Sec. 1).

    Offsets are returned in fine-level detector pixels (sigma_px per view) and
    the detector tilt psi in radians, with a step chosen so that a detector
    corner half_diag_px pixels from the centre moves sigma_px pixels per view.
    Returns float64 [K, 5].
    """
    rng = np.random.default_rng(seed)
    steps = rng.standard_normal((n_views, 5))
    steps[:, :4] *= sigma_px
    steps[:, 4] *= sigma_px / max(half_diag_px, 1.0)
    return np.cumsum(steps, axis=0)


def default_pitch(nu: int, src_axis_dist: float = 4 * R_HALF,
                  src_det_dist: float = 8 * R_HALF) -> float:
    """Detector pitch (world units) that makes nu pixels span the fan of the
    cylinder inscribed in the volume: 2 L tan(asin(R / D)) / nu."""
    return 2.0 * src_det_dist * math.tan(math.asin(R_HALF / src_axis_dist)) / nu


def ellipsoids(count: int, seed: int, centre_r: float = 0.35, centre_z: float = 0.35,
               axis_lo: float = 0.04, axis_hi: float = 0.2):
    """Random ellipsoid phantom description.

    Centres uniform in the cylinder r <= centre_r, |z| <= centre_z; semi-axes
    uniform in [axis_lo, axis_hi]; orientation from a uniform random unit
    quaternion; attenuation uniform in [0, 1), additive where ellipsoids overlap.
    Returns a dict of float64 arrays: centre [n,3] (x,y,z), axes [n,3],
    rot [n,3,3] (columns = body axes in world coordinates), mu [n].
    """
    rng = np.random.default_rng(seed)
    r = centre_r * np.sqrt(rng.random(count))
    phi = 2.0 * np.pi * rng.random(count)
    zc = centre_z * (2.0 * rng.random(count) - 1.0)
    centre = np.stack([r * np.cos(phi), r * np.sin(phi), zc], axis=1)
    axes = axis_lo + (axis_hi - axis_lo) * rng.random((count, 3))
    q = rng.standard_normal((count, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    rot = np.empty((count, 3, 3))
    rot[:, 0, 0] = 1 - 2 * (y * y + z * z)
    rot[:, 0, 1] = 2 * (x * y - z * w)
    rot[:, 0, 2] = 2 * (x * z + y * w)
    rot[:, 1, 0] = 2 * (x * y + z * w)
    rot[:, 1, 1] = 1 - 2 * (x * x + z * z)
    rot[:, 1, 2] = 2 * (y * z - x * w)
    rot[:, 2, 0] = 2 * (x * z - y * w)
    rot[:, 2, 1] = 2 * (y * z + x * w)
    rot[:, 2, 2] = 1 - 2 * (x * x + y * y)
    mu = rng.random(count)
    return {"centre": centre, "axes": axes, "rot": rot, "mu": mu}


def blobs(count: int, seed: int, sigma_lo: float, sigma_hi: float, centre_r: float = 0.25):
    """Isotropic Gaussian blobs amp * exp(-|x - c|^2 / (2 sigma^2)).

    Returns a dict of float64 arrays: centre [n,3], sigma [n], amp [n].
    """
    rng = np.random.default_rng(seed)
    centre = centre_r * (2.0 * rng.random((count, 3)) - 1.0)
    sigma = sigma_lo + (sigma_hi - sigma_lo) * rng.random(count)
    amp = 0.5 + rng.random(count)
    return {"centre": centre, "sigma": sigma, "amp": amp}


def _axis_centres(n: int, device, dtype):
    return (torch.arange(n, device=device, dtype=dtype) - (n - 1) / 2.0) / n


def voxelize_ellipsoids(ph: dict, n: int, supersample: int = 4, device="cpu",
                        dtype=torch.float64) -> torch.Tensor:
    """Voxel-mean of the additive ellipsoid phantom on an n^3 grid, by
    supersample^3 point samples per voxel.  Only each ellipsoid's bounding box
    is visited.  Returns [n][n][n] (z, y, x) of the given dtype.
    """
    vol = torch.zeros((n, n, n), device=device, dtype=torch.float64)
    s = supersample
    sub = ((torch.arange(s, device=device, dtype=torch.float64) + 0.5) / s - 0.5) / n
    h = 1.0 / n
    for c, ax, rot, mu in zip(ph["centre"], ph["axes"], ph["rot"], ph["mu"]):
        ext = float(ax.max())
        lo = np.floor((c - ext) * n + (n - 1) / 2.0).astype(int) - 1
        hi = np.ceil((c + ext) * n + (n - 1) / 2.0).astype(int) + 1
        lo = np.clip(lo, 0, n - 1)
        hi = np.clip(hi, 0, n - 1)
        if np.any(hi < lo):
            continue
        ix = torch.arange(lo[0], hi[0] + 1, device=device, dtype=torch.float64)
        iy = torch.arange(lo[1], hi[1] + 1, device=device, dtype=torch.float64)
        iz = torch.arange(lo[2], hi[2] + 1, device=device, dtype=torch.float64)
        # sample coordinates [nz*s][ny*s][nx*s]
        px = ((ix - (n - 1) / 2.0) * h)[:, None] + sub[None, :]
        py = ((iy - (n - 1) / 2.0) * h)[:, None] + sub[None, :]
        pz = ((iz - (n - 1) / 2.0) * h)[:, None] + sub[None, :]
        px = px.reshape(-1) - c[0]
        py = py.reshape(-1) - c[1]
        pz = pz.reshape(-1) - c[2]
        rt = torch.as_tensor(rot.T / ax[:, None], device=device)  # body coords / semi-axis
        # q = rt @ (x, y, z): evaluate as separable sums to avoid a huge 3-vector tensor
        acc = None
        for k in range(3):
            term = (rt[k, 0] * px[None, None, :] + rt[k, 1] * py[None, :, None]
                    + rt[k, 2] * pz[:, None, None])
            acc = term * term if acc is None else acc + term * term
        inside = (acc <= 1.0).to(torch.float64)
        occ = inside.reshape(len(iz), s, len(iy), s, len(ix), s).mean(dim=(1, 3, 5))
        vol[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] += float(mu) * occ
    return vol.to(dtype)


def voxelize_blobs(ph: dict, n: int, device="cpu", dtype=torch.float64) -> torch.Tensor:
    """Gaussian blobs sampled at voxel centres, [n][n][n] (z, y, x)."""
    c = _axis_centres(n, device, torch.float64)
    vol = torch.zeros((n, n, n), device=device, dtype=torch.float64)
    for cen, sg, amp in zip(ph["centre"], ph["sigma"], ph["amp"]):
        gx = torch.exp(-(c - cen[0]) ** 2 / (2 * sg * sg))
        gy = torch.exp(-(c - cen[1]) ** 2 / (2 * sg * sg))
        gz = torch.exp(-(c - cen[2]) ** 2 / (2 * sg * sg))
        vol += amp * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return vol.to(dtype)


def _gauss_blur3(x: torch.Tensor, sigma: float) -> torch.Tensor:
    """Separable Gaussian blur (zero padding) of a [n][n][n] float tensor."""
    rad = max(1, int(math.ceil(3.0 * sigma)))
    t = torch.arange(-rad, rad + 1, device=x.device, dtype=x.dtype)
    k = torch.exp(-t * t / (2 * sigma * sigma))
    k = k / k.sum()
    y = x[None, None]
    for dim in range(3):
        shape = [1, 1, 1, 1, 1]
        shape[2 + dim] = len(k)
        pad = [0, 0, 0, 0, 0, 0]
        pad[2 * (2 - dim)] = rad
        pad[2 * (2 - dim) + 1] = rad
        y = torch.nn.functional.conv3d(torch.nn.functional.pad(y, pad), k.view(shape))
    return y[0, 0]


def porous_texture(n: int, seed: int, device="cpu", solid: float = 0.3,
                   dtype=torch.float32) -> torch.Tensor:
    """Porous solid texture: white noise -> Gaussian blur (sigma 2 voxels of a
    256-voxel grid) -> normalise -> pores where the value exceeds 0.5 -> solid
    value `solid` inside r <= 0.45, |z| <= 0.45 -> blur (sigma 0.75 voxel).
    Returns [n][n][n] (z, y, x).
    """
    g = torch.Generator(device="cpu").manual_seed(seed)
    noise = torch.randn((n, n, n), generator=g, dtype=torch.float32).to(device)
    scale = n / 256.0
    f = _gauss_blur3(noise, 2.0 * scale)
    f = (f - f.mean()) / f.std()
    solid_mask = (f <= 0.5).to(torch.float32)
    c = _axis_centres(n, device, torch.float32)
    r2 = c[None, :, None] ** 2 + c[None, None, :] ** 2
    inside = (r2 <= 0.45 ** 2) & (c.abs()[:, None, None] <= 0.45)
    vol = solid * solid_mask * inside.to(torch.float32)
    vol = _gauss_blur3(vol, 0.75 * scale)
    return vol.to(dtype)


def poisson_log_data(b: torch.Tensor, photons: float, seed: int, chunk: int = 1 << 30) -> torch.Tensor:
    """Photon-counting noise on log data (Eq. 1): I ~ Poisson(I0 exp(-b)),
    returned as -ln(max(I, 1) / I0).  Works on any device; float32 result.
    Sinograms of more than `chunk` elements are drawn a block of whole views
    at a time (torch's Poisson sampler on the GPU gives wrong counts on
    tensors of more than 2^31 elements); smaller ones in one draw."""
    g = torch.Generator(device=b.device).manual_seed(seed)
    out = torch.empty(b.shape, dtype=torch.float32, device=b.device)
    per = max(1, chunk // max(1, b[0].numel())) if b.numel() > chunk else b.shape[0]
    for k0 in range(0, b.shape[0], per):
        lam = photons * torch.exp(-b[k0:k0 + per].to(torch.float32))
        counts = torch.poisson(lam, generator=g)
        out[k0:k0 + per] = -torch.log(torch.clamp(counts, min=1.0) / photons)
    return out


def random_indices(count: int, limits, seed: int) -> np.ndarray:
    """`count` random integer index tuples, each component in [0, limit)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, lim, size=count) for lim in limits], axis=1)


def random_volume(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Uniform [0, 1) random volume [n][n][n]."""
    return np.random.default_rng(seed).random((n, n, n)).astype(dtype)


def random_sino(k: int, nv: int, nu: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Standard-normal random sinogram [k][nv][nu]."""
    return np.random.default_rng(seed).standard_normal((k, nv, nu)).astype(dtype)
