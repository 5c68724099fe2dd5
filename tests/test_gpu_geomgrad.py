"""Differentiable form: the per-view geometry gradient kernel and the autograd
wrappers, against the FP64 oracle's analytic gradient (itself pinned by
central differences and by the closed-form Gaussian line integral)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2103_10329_gb300 import synth
from tests.helpers import TOL_F32, check_err, cuda, gpu_geom, oracle_scan, rel_err, scan_desc, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2103_10329_gb300 import build
    build.build()
    O.build()


# Geometry-gradient bound, per parameter type relative to that type's
# largest entry.  A view's gradient sums r_ray * dA_ray/dphi over its rays in
# float64, each ray's derivative summed along the ray in float32 from the
# bilinear gradient at the sample (a difference of neighbouring voxels).
# Float32 rounding of each term (~6e-8) and the sample positions' error
# (~1e-6 voxel, times the second difference of the smooth test volumes) give
# each ray's derivative a relative error e_ray ~ 1e-6; the sum over R rays
# of signed residuals cancels to ~sqrt(R) of a typical term while the errors
# add like sqrt(R) too, but with the full term size rather than the signed
# one, so the ratio is about e_ray * (rms |r D| / |mean r D|), up to ~1e2 for
# near-zero views of a type: 1e-4 of the type's largest entry.  The
# measured maxima are recorded beside it (MGCT_PARITY_REPORT).
GRAD_TOL = 1e-4


def smooth_volume(n, seed=5):
    return synth.voxelize_blobs(synth.blobs(4, seed, 0.06, 0.12, centre_r=0.2), n).numpy()


@pytest.mark.parametrize("tilt", [False, True])
def test_geometry_grad_vs_oracle(tilt):
    from paper_2103_10329_gb300 import mgct
    K, n, nu = 12, 40, 60
    drift = synth.drift_walk(K, 8, sigma_px=0.6, half_diag_px=40)
    if not tilt:
        drift[:, 4] = 0.0
    d = scan_desc(n, nu, nu, K, 2104, levels=1, drift=drift)
    g = gpu_geom(d)
    vol = smooth_volume(n)
    y = np.random.default_rng(3).standard_normal((K, nu, nu))
    ref = O.geometry_grad(oracle_scan(d), vol.astype(np.float32).astype(np.float64),
                          y.astype(np.float32).astype(np.float64))
    got = to_np(mgct.geometry_grad(g, cuda(vol), cuda(y)))
    # per parameter type, relative to that type's largest entry
    for j in range(5):
        check_err(np.abs(got[:, j] - ref[:, j]) / np.abs(ref[:, j]).max(), GRAD_TOL)


def test_view_subset_gradient():
    from paper_2103_10329_gb300 import mgct
    K, n, nu = 16, 32, 48
    drift = synth.drift_walk(K, 9, sigma_px=0.4, half_diag_px=30)
    d = scan_desc(n, nu, nu, K, 2104, levels=1, drift=drift)
    g = gpu_geom(d)
    vol = cuda(smooth_volume(n))
    y = cuda(np.random.default_rng(4).standard_normal((K, nu, nu)))
    full = mgct.geometry_grad(g, vol, y)
    sub = mgct.geometry_grad(g, vol, y[1::3].contiguous(), views=(1, len(range(1, K, 3)), 3))
    assert torch.allclose(sub, full[1::3], rtol=1e-12, atol=0)


def test_autograd_project_matches_oracle():
    from paper_2103_10329_gb300 import autograd as AG
    K, n, nu = 10, 32, 48
    drift = synth.drift_walk(K, 10, sigma_px=0.5, half_diag_px=30)
    d = scan_desc(n, nu, nu, K, 2104, levels=1, drift=drift)
    g = gpu_geom(d)
    vol_np = smooth_volume(n)
    y_np = np.random.default_rng(6).standard_normal((K, nu, nu)).astype(np.float32)
    vol = cuda(vol_np).requires_grad_(True)
    phi = torch.tensor(drift, dtype=torch.float64, device="cuda", requires_grad=True)
    loss = (AG.project(vol, g, phi) * cuda(y_np)).sum()
    loss.backward()
    og = O.level_geometry(oracle_scan(d), 0)
    ref_vol = O.backproject(og, y_np.astype(np.float64))
    ref_phi = O.geometry_grad(oracle_scan(d), vol_np.astype(np.float32).astype(np.float64), y_np.astype(np.float64))
    gv = to_np(vol.grad)
    # A^T of a signed sinogram: per voxel, relative to A^T |y| (the scale of
    # the sum's rounding error), as every back-projection test measures it
    ref_abs = O.backproject(og, np.abs(y_np).astype(np.float64))
    den = np.maximum(ref_abs, 1e-2 * ref_abs.max())
    check_err(np.abs(gv - ref_vol) / den, TOL_F32)
    gp = phi.grad.cpu().numpy()
    for j in range(5):
        check_err(np.abs(gp[:, j] - ref_phi[:, j]) / np.abs(ref_phi[:, j]).max(), GRAD_TOL)
    # the backward of the back-projection is the projection
    yy = cuda(y_np).requires_grad_(True)
    w = cuda(vol_np)
    (AG.backproject(yy, g) * w).sum().backward()
    ref_y = O.project(og, vol_np.astype(np.float32).astype(np.float64))
    check_err(rel_err(to_np(yy.grad), ref_y), TOL_F32)


def test_joint_estimation_recovers_detector_offset():
    """Sec. 1 motivates estimating drift jointly with the image.  Data made
    with every view's detector shifted by 1.5 pixels along u; starting from no
    drift, alternating multigrid iterations on mu with gradient steps on a
    shared offset through the autograd projector recovers the shift."""
    from paper_2103_10329_gb300 import autograd as AG
    from paper_2103_10329_gb300 import mgct
    K, n, nu = 40, 32, 48
    true = np.zeros((K, 5))
    true[:, 2] = 1.5
    d_true = scan_desc(n, nu, nu, K, 2104, levels=2, drift=true)
    truth = smooth_volume(n, seed=11)
    b = cuda(O.project(O.level_geometry(oracle_scan(d_true), 0), truth))
    g = gpu_geom(scan_desc(n, nu, nu, K, 2104, levels=2))
    rec = mgct.Reconstructor(g)
    off = 0.0
    vol = torch.zeros((n, n, n), device="cuda")
    errs = []
    for outer in range(6):
        phi_np = np.zeros((K, 5))
        phi_np[:, 2] = off
        g.set_drift(phi_np)
        rec.prepare(b)
        for _ in range(2):
            rec.iterate(vol)
        for _ in range(3):
            phi = torch.tensor(phi_np, device="cuda", requires_grad=True)
            r = AG.project(vol, g, phi) - b
            loss = 0.5 * (r * r).sum()
            loss.backward()
            gsum = float(phi.grad[:, 2].sum())
            # Gauss-Newton step on the shared offset: curvature from a secant
            eps = 0.05
            p2 = phi_np.copy()
            p2[:, 2] += eps
            phi2 = torch.tensor(p2, device="cuda", requires_grad=True)
            r2 = AG.project(vol, g, phi2) - b
            (0.5 * (r2 * r2).sum()).backward()
            curv = (float(phi2.grad[:, 2].sum()) - gsum) / eps
            if curv > 0:
                off -= gsum / curv
            phi_np[:, 2] = off
        errs.append(abs(off - 1.5))
    assert errs[-1] < 0.2 * 1.5, errs
    assert errs[-1] < errs[0], errs


def test_geometry_grad_full_size_sampled():
    """The drift-estimation workload at full size (256^3, 384^2 detector, 720
    views with source/detector offsets and tilt as Gaussian random walks of
    0.3 px per view): the gradient of all views in one call, checked at
    sampled views against the oracle (each view's gradient depends on that
    view alone, so the oracle runs on a scan of just those views)."""
    from paper_2103_10329_gb300 import mgct
    K, n, nu = 720, 256, 384
    drift = synth.drift_walk(K, 31, sigma_px=0.3, half_diag_px=0.5 * np.sqrt(2.0) * nu)
    d = scan_desc(n, nu, nu, K, 2104, levels=1, drift=drift)
    g = gpu_geom(d)
    vol = synth.voxelize_blobs(synth.blobs(6, 7, 0.05, 0.15, centre_r=0.25), n).numpy().astype(np.float32)
    y = torch.randn((K, nu, nu), device="cuda", generator=torch.Generator("cuda").manual_seed(9))
    got = to_np(mgct.geometry_grad(g, cuda(vol), y))
    views = np.array([0, 233, 500, 719])
    ds = dict(d, theta=d["theta"][views], z=d["z"][views], drift=drift[views])
    ref = O.geometry_grad(oracle_scan(ds), vol.astype(np.float64), to_np(y[torch.as_tensor(views, device="cuda")]))
    for j in range(5):
        check_err(np.abs(got[views, j] - ref[:, j]) / np.abs(ref[:, j]).max(), GRAD_TOL)


def test_joint_estimation_recovers_per_view_drift():
    """Every view drifts (source and detector offsets along both detector
    axes and the detector tilt, Gaussian random walks of 0.3 px per view, as
    in the drift workload).  Starting from no drift, the alternation of
    multigrid iterations with Newton steps built on the geometry gradient
    recovers what the data determine: the tilt and the projection shift along
    u of the volume centre (ds_u + dd_u at magnification 2) to a small
    fraction of the drift, every parameter type better than no correction,
    and an image much closer to the phantom than without the correction.
    (A source and a detector shift cancelling at the centre, and a vertical
    offset common to all views, which equals moving the object, are pinned
    only weakly or not at all.)"""
    from paper_2103_10329_gb300 import joint, mgct
    K, n, nu = 90, 64, 96
    half = 0.5 * np.sqrt(2.0) * nu
    true = synth.drift_walk(K, 41, sigma_px=0.3, half_diag_px=half)
    d_true = scan_desc(n, nu, nu, K, 2104, levels=2, drift=true)
    truth = smooth_volume(n, seed=12)
    gt = gpu_geom(d_true)
    b = mgct.project(gt, cuda(truth))
    gt.close()
    g = gpu_geom(scan_desc(n, nu, nu, K, 2104, levels=2))
    mu, phi, hist = joint.estimate(g, b, half, schedule=((1, 3), (0, 3)), truth_phi=true)
    err = phi - true
    rms0 = np.sqrt(np.mean(true ** 2, axis=0))
    rms1 = np.sqrt(np.mean(err ** 2, axis=0))
    shift0 = np.sqrt(np.mean((true[:, 0] + true[:, 2]) ** 2))
    shift1 = np.sqrt(np.mean((err[:, 0] + err[:, 2]) ** 2))
    assert rms1[4] < 0.25 * rms0[4], (rms0.tolist(), rms1.tolist(), hist)
    assert shift1 < 0.25 * shift0, (shift0, shift1, hist)
    assert np.all(rms1 < rms0), (rms0.tolist(), rms1.tolist())
    g.set_drift(None)
    rec = mgct.Reconstructor(g)
    rec.prepare(b)
    mu0 = torch.zeros_like(mu)
    for _ in range(2 * (3 + 3 + 1)):
        rec.iterate(mu0)
    t = cuda(truth)
    e_est = float(torch.sqrt(torch.mean((mu - t) ** 2)))
    e_none = float(torch.sqrt(torch.mean((mu0 - t) ** 2)))
    assert e_est < 0.5 * e_none, (e_est, e_none)
    print(f"\njoint estimation: drift rms {rms0.round(3).tolist()} -> {rms1.round(3).tolist()}; u shift "
          f"{shift0:.3f} -> {shift1:.3f} px; image rmse {e_none:.4g} -> {e_est:.4g}")
