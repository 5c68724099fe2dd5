"""Pins for the FP64 oracle: closed forms, invariants, brute force and special
cases that reduce to library routines.  CPU only."""
import math
import os

import numpy as np
import pytest
import scipy.ndimage

import oracle as O
from paper_2103_10329_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def make_scan(n, nviews=12, seed=1, drift=None, nu=None, nv=None, flat_z=False):
    th, z = synth.trajectory(nviews, seed)
    nu = nu or int(round(1.5 * n))
    nv = nv or nu
    if flat_z:
        z = np.zeros_like(z)
    return O.Scan(n=n, nu=nu, nv=nv, theta=th, z=z, pitch=synth.default_pitch(nu), drift=drift)


# ---------------------------------------------------------------- geometry

def test_geometry_conventions():
    """Sec. 2: distances are measured from the source; the detector is flat and
    faces the source; its pixel grid is centred on the source-axis line."""
    scan = make_scan(16, nviews=7)
    g = O.level_geometry(scan, 0)
    for k in range(g.n_views):
        s = g.src[k]
        assert math.isclose(math.hypot(s[0], s[1]), 2.0, rel_tol=1e-14)
        assert math.isclose(s[2], scan.z[k], abs_tol=1e-15)
        centre = g.det[k] + 0.5 * (g.nu - 1) * g.pu[k] + 0.5 * (g.nv - 1) * g.pv[k]
        v = centre - s
        assert math.isclose(np.linalg.norm(v), 4.0, rel_tol=1e-14)
        # the detector centre lies on the line from the source through the rotation axis
        assert abs(v[2]) < 1e-14 and abs(s[0] * v[1] - s[1] * v[0]) < 1e-12
        assert s[0] * v[0] + s[1] * v[1] < 0
        # pixel steps orthogonal to each other and to the viewing direction
        assert abs(np.dot(g.pu[k], g.pv[k])) < 1e-15
        assert abs(np.dot(g.pu[k], v)) < 1e-13 and abs(np.dot(g.pv[k], v)) < 1e-13
        assert math.isclose(np.linalg.norm(g.pu[k]), scan.pitch, rel_tol=1e-14)


def test_geometry_drift_moves_source_and_detector():
    drift = np.zeros((5, 5))
    drift[:, 0] = 1.0   # source +1 pixel along u
    drift[:, 3] = -2.0  # detector -2 pixels along v
    drift[:, 4] = 0.1   # tilt
    scan0 = make_scan(16, nviews=5)
    scan1 = make_scan(16, nviews=5, drift=drift)
    g0, g1 = O.level_geometry(scan0, 0), O.level_geometry(scan1, 0)
    eu = g0.pu / scan0.pitch
    ev = g0.pv / scan0.pitch
    np.testing.assert_allclose(g1.src - g0.src, eu * scan0.pitch, atol=1e-15)
    c0 = g0.det + 0.5 * (g0.nu - 1) * g0.pu + 0.5 * (g0.nv - 1) * g0.pv
    c1 = g1.det + 0.5 * (g1.nu - 1) * g1.pu + 0.5 * (g1.nv - 1) * g1.pv
    np.testing.assert_allclose(c1 - c0, -2.0 * ev * scan0.pitch, atol=1e-14)
    cosang = np.sum(g1.pu * g0.pu, axis=1) / scan0.pitch ** 2
    np.testing.assert_allclose(cosang, math.cos(0.1), rtol=1e-14)


def test_coarse_grid_pixels_are_fine_pixel_means():
    """Restricted data (2x2 mean) sits at the centre of its four fine pixels."""
    scan = make_scan(16, nviews=3)
    g0, g1 = O.level_geometry(scan, 0), O.level_geometry(scan, 1)
    for k in range(3):
        p0 = O.pixel_centres(g0, k)
        p1 = O.pixel_centres(g1, k)
        mean = p0.reshape(g1.nv, 2, g1.nu, 2, 3).mean(axis=(1, 3))
        np.testing.assert_allclose(p1, mean, atol=1e-14)


# ---------------------------------------------------------------- P (= A)

def test_blob_integrals_second_order():
    """Gaussian blob: closed-form line integral amp sigma sqrt(2 pi) exp(-d^2/2s^2).
    Joseph's bilinear sampling is second order: the error falls ~4x per
    doubling of N once sigma >= 3h."""
    th, z = synth.trajectory(10, 3)
    drift = synth.drift_walk(10, 4, sigma_px=0.5, half_diag_px=20)
    ph = synth.blobs(3, 5, 0.07, 0.1, centre_r=0.12)
    errs = []
    for n in (32, 64, 128):
        nu = int(1.5 * n)
        scan = O.Scan(n=n, nu=nu, nv=nu, theta=th, z=0.2 * z, pitch=synth.default_pitch(nu),
                      drift=drift)
        g = O.level_geometry(scan, 0)
        vol = synth.voxelize_blobs(ph, n).numpy()
        a = O.project(g, vol)
        ex = O.blob_line_integrals(g, ph)
        errs.append(np.abs(a - ex).max() / np.abs(ex).max())
    assert errs[-1] < 2e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def test_ellipsoid_chords_converge():
    """Analytic ellipsoid chords vs P of the supersampled voxelisation: the
    mean error falls under refinement (edges make it first order)."""
    th, z = synth.trajectory(6, 7)
    ph = synth.ellipsoids(4, 8, axis_lo=0.08, axis_hi=0.2)
    errs = []
    for n in (16, 32, 64):
        nu = int(1.5 * n)
        scan = O.Scan(n=n, nu=nu, nv=nu, theta=th, z=0.5 * z, pitch=synth.default_pitch(nu))
        g = O.level_geometry(scan, 0)
        vol = synth.voxelize_ellipsoids(ph, n, supersample=4).numpy()
        a = O.project(g, vol)
        ex = O.ellipsoid_line_integrals(g, ph)
        errs.append(np.abs(a - ex).mean() / np.abs(ex).mean())
    # at least first-order convergence (edges), measured ~2.5x per doubling
    assert errs[0] / errs[1] > 1.8 and errs[1] / errs[2] > 1.8, errs


def _single_view(src, det, pu, pv, n, nu=1, nv=1):
    return O.LevelGeom(n, nu, nv, 1.0 / n, np.array([src], float), np.array([det], float),
                       np.array([pu], float), np.array([pv], float))


@pytest.mark.parametrize("axis", [0, 1])
def test_axis_aligned_ray_constant_volume(axis):
    """A ray along a volume axis through voxel centres of a constant volume
    samples every plane at a voxel centre: integral = N h = 1 exactly."""
    n = 8
    h = 1.0 / n
    yc, zc = (2 - (n - 1) / 2) * h, (5 - (n - 1) / 2) * h
    if axis == 0:
        src, det = [2.0, yc, zc], [-2.0, yc, zc]
        pu = [0.0, 0.01, 0.0]
    else:
        src, det = [yc, 2.0, zc], [yc, -2.0, zc]
        pu = [0.01, 0.0, 0.0]
    g = _single_view(src, det, pu, [0, 0, 0.01], n)
    a = O.project(g, np.ones((n, n, n)))
    assert a.shape == (1, 1, 1)
    assert abs(a[0, 0, 0] - 1.0) < 1e-14
    # and a ray through one row of voxels picks out that row only
    vol = np.zeros((n, n, n))
    if axis == 0:
        vol[5, 2, :] = np.arange(n) + 1.0
    else:
        vol[5, :, 2] = np.arange(n) + 1.0
    assert abs(O.project(g, vol)[0, 0, 0] - h * n * (n + 1) / 2) < 1e-13


def test_dense_matrix_matches_entry_weights_and_transpose():
    """Brute force at 8^3: the matrix assembled column by column from P e_j
    equals the per-entry weight function; B e_i rows equal its transpose."""
    n = 8
    drift = synth.drift_walk(4, 11, sigma_px=0.7, half_diag_px=6)
    scan = make_scan(n, nviews=4, seed=2, drift=drift, nu=12, nv=10)
    g = O.level_geometry(scan, 0)
    nvox = n ** 3
    nray = g.n_views * g.nv * g.nu
    A = np.zeros((nray, nvox))
    for j in range(nvox):
        e = np.zeros(nvox)
        e[j] = 1.0
        A[:, j] = O.project(g, e.reshape(n, n, n)).ravel()
    W = np.zeros_like(A)
    for k in range(g.n_views):
        for jv in range(g.nv):
            for ju in range(g.nu):
                row = (k * g.nv + jv) * g.nu + ju
                for iz in range(n):
                    for iy in range(n):
                        for ix in range(n):
                            W[row, (iz * n + iy) * n + ix] = O.weight(g, k, ju, jv, ix, iy, iz)
    assert np.count_nonzero(A) > 1000
    np.testing.assert_allclose(A, W, rtol=0, atol=1e-14)
    rng = np.random.default_rng(0)
    for row in rng.choice(nray, 20, replace=False):
        e = np.zeros(nray)
        e[row] = 1.0
        bt = O.backproject(g, e.reshape(g.n_views, g.nv, g.nu)).ravel()
        np.testing.assert_allclose(bt, A[row], rtol=0, atol=1e-14)


# ---------------------------------------------------------------- B (= A^T)

def test_adjoint_identity():
    """Sec. 2.1: B is the adjoint of P.  <Px, y> = <x, By> to 1e-12."""
    n = 24
    drift = synth.drift_walk(9, 12, sigma_px=0.5, half_diag_px=18)
    scan = make_scan(n, nviews=9, seed=3, drift=drift)
    g = O.level_geometry(scan, 0)
    x = synth.random_volume(n, 1)
    y = synth.random_sino(g.n_views, g.nv, g.nu, 2)
    lhs = float(np.vdot(O.project(g, x), y))
    rhs = float(np.vdot(x, O.backproject(g, y)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), np.abs(x).sum())


def test_backproject_voxels_matches_scatter():
    n = 16
    scan = make_scan(n, nviews=6, seed=4)
    g = O.level_geometry(scan, 0)
    y = synth.random_sino(g.n_views, g.nv, g.nu, 3)
    full = O.backproject(g, y)
    vox = synth.random_indices(40, (n, n, n), 5)
    got = O.backproject_voxels(g, y, vox, radius=4)
    want = full[vox[:, 2], vox[:, 1], vox[:, 0]]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_project_rays_matches_full():
    n = 16
    scan = make_scan(n, nviews=5, seed=6)
    g = O.level_geometry(scan, 0)
    x = synth.random_volume(n, 7)
    full = O.project(g, x)
    rays = synth.random_indices(50, (g.n_views, g.nv, g.nu), 8)
    got = O.project_rays(g, x, rays)
    np.testing.assert_allclose(got, full[rays[:, 0], rays[:, 1], rays[:, 2]], rtol=1e-14)


# ---------------------------------------------------------------- p (Eq. 5)

def _golden_eq5():
    rows = []
    with open(os.path.join(GOLDEN, "eq5_kernel.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return np.array(rows).reshape(3, 3, 3) / 64.0


def test_eq5_coefficients_and_invariants():
    k = _golden_eq5()
    np.testing.assert_array_equal(O.EQ5, k)
    assert k.sum() == 0.0                       # zero DC response (Sec. 3 discussion)
    assert abs(np.abs(k).sum() - 2.0) < 1e-15
    assert np.array_equal(k, k[::-1, ::-1, ::-1])
    assert np.array_equal(k, np.transpose(k, (0, 2, 1)))
    # Fourier symbol: real, in [0, 1.625], 0 at DC, 1.625 at (pi along an in-slice axis)
    big = np.zeros((64, 64, 64))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                big[(dz - 1) % 64, (dy - 1) % 64, (dx - 1) % 64] = k[dz, dy, dx]
    sym = np.fft.fftn(big)
    assert np.abs(sym.imag).max() < 1e-13
    assert abs(sym.real.min()) < 1e-13 and sym.real.min() > -1e-13
    assert abs(sym.real.max() - 1.625) < 1e-13
    assert abs(sym.real[0, 0, 32] - 1.625) < 1e-13


@pytest.mark.parametrize("axis", [2, 0])
def test_precondition_equals_library_correlation(axis):
    """p * x with zero padding equals scipy's constant-mode correlation with
    the Eq. 5 kernel (a symmetric kernel: convolution = correlation); the
    outer index runs along the chosen slice axis."""
    x = synth.random_volume(11, 9)
    k = O.eq5_kernel(axis)
    want = scipy.ndimage.correlate(x, k, mode="constant", cval=0.0)
    np.testing.assert_allclose(O.precondition(x, axis), want, atol=1e-13)
    # impulse response in the interior reproduces the kernel with its orientation
    d = np.zeros((7, 7, 7))
    d[3, 3, 3] = 1.0
    resp = O.precondition(d, axis)[2:5, 2:5, 2:5]
    np.testing.assert_allclose(resp, k, atol=1e-15)
    if axis == 2:
        assert resp[1, 1, 1] == 1.0 and resp[0, 1, 1] == 0.0 and resp[1, 0, 1] == -4 / 64


def test_precondition_self_adjoint():
    x = synth.random_volume(10, 1)
    y = synth.random_volume(10, 2)
    assert abs(np.vdot(x, O.precondition(y)) - np.vdot(O.precondition(x), y)) < 1e-12


def test_soft_threshold():
    x = np.array([-2.0, -0.5, 0.0, 0.3, 1.5])
    np.testing.assert_allclose(O.soft_threshold(x, 0.5), [-1.5, 0.0, 0.0, 0.0, 1.0])
    np.testing.assert_array_equal(O.soft_threshold(x, 0.0), x)


# ---------------------------------------------------------------- R / P

def test_restrict_prolong_invariants():
    n = 8
    c = np.full((n, n, n), 3.25)
    np.testing.assert_allclose(O.restrict_volume(np.full((2 * n,) * 3, 3.25)), c)
    np.testing.assert_allclose(O.prolong(c), np.full((2 * n,) * 3, 3.25))
    # restrict of a fine linear function = the linear function at coarse centres
    nf = 16
    i = np.arange(nf)
    xf = (i - (nf - 1) / 2) / nf
    lin_f = 0.3 * xf[None, None, :] - 1.7 * xf[None, :, None] + 0.9 * xf[:, None, None]
    ic = np.arange(nf // 2)
    xc = (ic - (nf // 2 - 1) / 2) / (nf // 2)
    lin_c = 0.3 * xc[None, None, :] - 1.7 * xc[None, :, None] + 0.9 * xc[:, None, None]
    np.testing.assert_allclose(O.restrict_volume(lin_f), lin_c, atol=1e-14)
    # prolongation is exact for linear functions away from the clamped edges
    pf = O.prolong(lin_c)
    np.testing.assert_allclose(pf[1:-1, 1:-1, 1:-1], lin_f[1:-1, 1:-1, 1:-1], atol=1e-14)
    # the 1-D stencil: fine cells 2i, 2i+1 take 3/4 of coarse i and 1/4 of i-1, i+1
    c1 = np.zeros((4, 4, 4))
    c1[1, 1, 1] = 1.0
    p1 = O.prolong(c1)
    assert abs(p1[2, 2, 2] - 0.75 ** 3) < 1e-15
    assert abs(p1[1, 2, 2] - 0.25 * 0.75 ** 2) < 1e-15
    assert abs(p1[4, 2, 2] - 0.25 * 0.75 ** 2) < 1e-15
    assert p1[0, 2, 2] == 0.0
    b = synth.random_sino(3, 8, 6, 1)
    rb = O.restrict_sino(b)
    assert rb.shape == (3, 4, 3)
    assert abs(rb[1, 2, 1] - b[1, 4:6, 2:4].mean()) < 1e-15


# ---------------------------------------------------------------- solvers

def _dense(g):
    n = g.n
    A = np.zeros((g.n_views * g.nv * g.nu, n ** 3))
    for j in range(n ** 3):
        e = np.zeros(n ** 3)
        e[j] = 1.0
        A[:, j] = O.project(g, e.reshape(n, n, n)).ravel()
    return A


def test_landweber_line_search_and_fixed_point():
    """Eq. 2/4 with the exact line search: alpha minimises |b - P(mu + alpha d)|
    along d, the predicted residual is the true one, and the least-squares
    solution (numpy lstsq on the dense matrix) is a fixed point of SIRT."""
    n = 6
    scan = make_scan(n, nviews=16, seed=9, nu=10, nv=10)
    g = O.level_geometry(scan, 0)
    A = _dense(g)
    x_true = synth.random_volume(n, 3)
    b = (A @ x_true.ravel()).reshape(g.n_views, g.nv, g.nu) + 0.01 * synth.random_sino(
        g.n_views, g.nv, g.nu, 4)
    mu = np.zeros((n, n, n))
    prev = None
    for precond in (True, False):
        mu = np.zeros((n, n, n))
        for it in range(5):
            new, st = O.landweber_step(g, mu, b, precond=precond)
            r_new = np.sum((b - O.project(g, new)) ** 2)
            assert abs(r_new - st["r2_pred"]) <= 1e-9 * st["r2"]
            assert r_new <= st["r2"] * (1 + 1e-12)
            d = (new - mu) / st["alpha"] if st["alpha"] != 0 else None
            if d is not None:
                for eps in (1e-3, -1e-3):
                    alt = np.sum((b - O.project(g, mu + (st["alpha"] * (1 + eps)) * d)) ** 2)
                    assert alt >= r_new * (1 - 1e-12)
            mu = new
    xs, *_ = np.linalg.lstsq(A, b.ravel(), rcond=None)
    xs = xs.reshape(n, n, n)
    out, st = O.landweber_step(g, xs, b, precond=False, alpha=0.5)
    np.testing.assert_allclose(out, xs, atol=1e-9)


def test_sirt_converges_to_least_squares():
    """Brute force at 4^3: SIRT (Eq. 2) with a fixed alpha < 2 / |A|^2 converges
    to numpy's least-squares solution."""
    n = 4
    scan = make_scan(n, nviews=10, seed=10, nu=6, nv=6)
    g = O.level_geometry(scan, 0)
    A = _dense(g)
    lmax = np.linalg.norm(A, 2) ** 2
    x_true = synth.random_volume(n, 5)
    b = (A @ x_true.ravel()).reshape(g.n_views, g.nv, g.nu) + 0.01 * synth.random_sino(
        g.n_views, g.nv, g.nu, 6)
    xs, *_ = np.linalg.lstsq(A, b.ravel(), rcond=None)
    mu = np.zeros((n, n, n))
    s = np.linalg.svd(A, compute_uv=False)
    iters = int(np.ceil(30.0 / (1.9 * (s[-1] ** 2) / lmax)))
    iters = min(iters, 20000)
    for _ in range(iters):
        mu, _ = O.landweber_step(g, mu, b, alpha=1.9 / lmax, precond=False)
    assert np.abs(mu.ravel() - xs).max() < 1e-6 * np.abs(xs).max()


def test_osemtr_fixed_point_and_direction():
    """Eq. 3: with consistent data b = P x, x is a fixed point (numerator 0);
    from below (mu = 0.5 x) one pass moves mu towards x."""
    n = 12
    scan = make_scan(n, nviews=16, seed=11)
    g = O.level_geometry(scan, 0)
    x = 0.5 * synth.random_volume(n, 8) + 0.2
    b = O.project(g, x)
    out = O.osemtr_pass(g, x, b, n_subsets=4)
    assert np.abs(out - x).max() < 1e-12
    mu0 = 0.5 * x
    mu1 = O.osemtr_pass(g, mu0, b, n_subsets=4)
    r0 = np.linalg.norm(b - O.project(g, mu0))
    r1 = np.linalg.norm(b - O.project(g, mu1))
    assert r1 < 0.5 * r0


def _dense_from_weights(g):
    """A as a dense matrix from the per-entry weight function alone (rows
    (view, v, u), columns (z, y, x)), independent of the projector's loops."""
    n = g.n
    A = np.zeros((g.n_views * g.nv * g.nu, n ** 3))
    for k in range(g.n_views):
        for jv in range(g.nv):
            for ju in range(g.nu):
                row = (k * g.nv + jv) * g.nu + ju
                for iz in range(n):
                    for iy in range(n):
                        for ix in range(n):
                            A[row, (iz * n + iy) * n + ix] = O.weight(g, k, ju, jv, ix, iy, iz)
    return A


@pytest.mark.parametrize("m_sub", [1, 3])
def test_osemtr_pass_brute_force(m_sub):
    """Eq. 3 written out with a dense A from the per-entry weights at 5^3,
    subset by subset (views k = m mod M, in order m = 0..M-1):
    mu += A_m^T (exp(-A_m mu) - exp(-b_m)) / A_m^T (exp(-A_m mu) A_m 1),
    where the denominator exceeds 1e-12 of its maximum; the oracle's pass
    (projector and scatter loops) must agree to 1e-12."""
    n, k = 5, 6
    scan = make_scan(n, nviews=k, seed=21, nu=8, nv=8)
    g = O.level_geometry(scan, 0)
    A = _dense_from_weights(g)
    x = 0.6 * synth.random_volume(n, 22) + 0.1
    b = (A @ x.ravel()) * 1.05 + 0.01
    mu0 = 0.5 * synth.random_volume(n, 23) + 0.2
    got = O.osemtr_pass(g, mu0, b.reshape(k, g.nv, g.nu), n_subsets=m_sub)
    mu = mu0.ravel().copy()
    rows_per_view = g.nv * g.nu
    for m in range(m_sub):
        rows = np.concatenate([np.arange(v * rows_per_view, (v + 1) * rows_per_view) for v in range(m, k, m_sub)])
        Am = A[rows]
        t = np.exp(-(Am @ mu))
        num = Am.T @ (t - np.exp(-b[rows]))
        den = Am.T @ (t * (Am @ np.ones(n ** 3)))
        mask = den > 1e-12 * den.max()
        mu[mask] += num[mask] / den[mask]
    assert np.abs(mu - mu0.ravel()).max() > 1e-3  # the pass moved mu
    np.testing.assert_allclose(got.ravel(), mu, rtol=0, atol=1e-12)


def test_landweber_step_brute_force():
    """Eq. 4 written out with the dense A at 5^3 and Eq. 5 as a dense 27-point
    operator: d = p (A^T (b - A mu)), alpha = <r, A d> / |A d|^2,
    mu + alpha d; the oracle's step must agree to 1e-12."""
    n, k = 5, 5
    scan = make_scan(n, nviews=k, seed=24, nu=8, nv=8)
    g = O.level_geometry(scan, 0)
    A = _dense_from_weights(g)
    mu0 = synth.random_volume(n, 25)
    b = A @ synth.random_volume(n, 26).ravel()
    got, st = O.landweber_step(g, mu0, b.reshape(k, g.nv, g.nu))
    P = _dense_eq5(n)
    r = b - A @ mu0.ravel()
    d = P @ (A.T @ r)
    ad = A @ d
    alpha = float(r @ ad) / float(ad @ ad)
    assert abs(st["alpha"] - alpha) <= 1e-12 * abs(alpha)
    np.testing.assert_allclose(got.ravel(), mu0.ravel() + alpha * d, rtol=0, atol=1e-12)


def test_multigrid_single_level_is_one_landweber_step():
    n = 8
    scan = make_scan(n, nviews=6, seed=12)
    g = O.level_geometry(scan, 0)
    x = synth.random_volume(n, 9)
    b = O.project(g, x)
    mu0 = 0.1 * synth.random_volume(n, 10)
    mg = O.multigrid(scan, mu0, [b], levels=1)
    lw, _ = O.landweber_step(g, mu0, b)
    np.testing.assert_allclose(mg, lw, rtol=0, atol=1e-13)


def test_multigrid_structure_two_levels():
    """Alg. 1 with two grids: the fine estimate after the coarse correction is
    mu + Prolongate(osemtr(R mu) - R mu), then one Landweber step."""
    n = 8
    scan = make_scan(n, nviews=8, seed=13)
    x = synth.random_volume(n, 11)
    b = O.project(O.level_geometry(scan, 0), x)
    bl = O.data_levels(b, 2)
    mu0 = 0.2 * synth.random_volume(n, 12)
    got = O.multigrid(scan, mu0, bl, levels=2)
    mc = O.restrict_volume(mu0)
    mc2 = O.osemtr_pass(O.level_geometry(scan, 1), mc, bl[1])
    want, _ = O.landweber_step(O.level_geometry(scan, 0), mu0 + O.prolong(mc2 - mc), b)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def _dense_eq5(n):
    """Eq. 5 (z slices) as a dense n^3 x n^3 correlation with zero padding."""
    kern = O.eq5_kernel(2)
    P = np.zeros((n ** 3, n ** 3))
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            z, y, x = iz + dz, iy + dy, ix + dx
                            if 0 <= z < n and 0 <= y < n and 0 <= x < n:
                                P[(iz * n + iy) * n + ix, (z * n + y) * n + x] = kern[dz + 1, dy + 1, dx + 1]
    return P


def _dense_prolong_1d(nc):
    """Cell-centred linear interpolation to 2 nc cells: fine cell f sits at
    coarse coordinate f/2 - 1/4, between its two nearest coarse centres
    (weights 3/4 and 1/4), the outer neighbour clamped at the edges."""
    M = np.zeros((2 * nc, nc))
    for f in range(2 * nc):
        i, near = divmod(f, 2)
        other = min(max(i + (1 if near else -1), 0), nc - 1)
        M[f, i] += 0.75
        M[f, other] += 0.25
    return M


@pytest.mark.parametrize("levels,fas", [(2, False), (3, False), (3, True)])
def test_multigrid_brute_force(levels, fas):
    """Two iterations of Alg. 1 written out with dense operators at 8^3 (grids
    8, 4 and 2): A per grid from the per-entry weights, restriction as 2x2x2
    and 2x2 means, prolongation as the Kronecker product of the 1-D cell-
    centred interpolation, Eq. 5 as a dense stencil, OS-EMTR on the coarsest
    grid (8 subsets, one view each) and the line-searched Landweber step on
    every other grid.  With fas the coarse data are R (b - A mu) + A_c R mu
    instead of R b.  The oracle's multigrid must agree to 1e-11."""
    n, k = 8, 8
    scan = make_scan(n, nviews=k, seed=27, nu=12, nv=12)
    A = [_dense_from_weights(O.level_geometry(scan, l)) for l in range(levels)]
    sizes = [(n >> l, 12 >> l) for l in range(levels)]

    def restrict_vol(m):
        R = np.zeros((m ** 3 // 8, m ** 3))
        h = m // 2
        for z in range(m):
            for y in range(m):
                for x in range(m):
                    R[((z // 2) * h + y // 2) * h + x // 2, (z * m + y) * m + x] = 1.0 / 8
        return R

    def restrict_sino(d):
        R = np.zeros((k * (d // 2) ** 2, k * d * d))
        h = d // 2
        for v in range(k):
            for jv in range(d):
                for ju in range(d):
                    R[(v * h + jv // 2) * h + ju // 2, (v * d + jv) * d + ju] = 0.25
        return R

    def landweber(l, mu, b):
        P = _dense_eq5(sizes[l][0])
        r = b - A[l] @ mu
        dd = P @ (A[l].T @ r)
        ad = A[l] @ dd
        den = float(ad @ ad)
        return mu + (float(r @ ad) / den if den > 0 else 0.0) * dd

    def osemtr(l, mu, b):
        mu = mu.copy()
        rows_per_view = sizes[l][1] ** 2
        pi = A[l] @ np.ones(A[l].shape[1])
        for m in range(8):
            rows = np.arange(m * rows_per_view, (m + 1) * rows_per_view)
            Am = A[l][rows]
            t = np.exp(-(Am @ mu))
            num = Am.T @ (t - np.exp(-b[rows]))
            den = Am.T @ (t * pi[rows])
            mask = den > 1e-12 * den.max()
            mu[mask] += num[mask] / den[mask]
        return mu

    x = synth.random_volume(n, 28)
    b = [A[0] @ x.ravel()]
    for l in range(1, levels):
        b.append(restrict_sino(sizes[l - 1][1]) @ b[-1])

    def mg(l, mu, bl):
        if l + 1 < levels:
            mc = restrict_vol(sizes[l][0]) @ mu
            bc = restrict_sino(sizes[l][1]) @ (bl - A[l] @ mu) + A[l + 1] @ mc if fas else b[l + 1]
            mc_new = mg(l + 1, mc, bc) if l + 1 < levels - 1 else osemtr(l + 1, mc, bc)
            p1 = _dense_prolong_1d(sizes[l + 1][0])
            mu = mu + np.kron(np.kron(p1, p1), p1) @ (mc_new - mc)
        return landweber(l, mu, bl)

    mu = np.zeros(n ** 3)
    for _ in range(2):
        mu = mg(0, mu, b[0])
    got = O.reconstruct(scan, b[0].reshape(k, 12, 12), iters=2, levels=levels, fas=fas)
    assert np.abs(mu).max() > 0.1
    np.testing.assert_allclose(got.ravel(), mu, rtol=0, atol=1e-11)


def test_precondition_custom_kernel():
    """A kernel given in place of Eq. 5 is applied as the correlation
    out(p) = sum_d k[d] x(p + d) (scipy's `correlate`, zero padding); Eq. 5
    itself passed as the kernel reproduces the default."""
    x = synth.random_volume(9, 60) - 0.5
    k = np.random.default_rng(61).standard_normal((3, 3, 3))
    np.testing.assert_allclose(O.precondition(x, kernel=k), scipy.ndimage.correlate(x, k, mode="constant"),
                               rtol=0, atol=1e-13)
    np.testing.assert_allclose(O.precondition(x, kernel=O.eq5_kernel(2)), O.precondition(x), rtol=0, atol=0)


# ---------------------------------------------------------------- bilateral filter (Alg. 1)

def test_bilateral_brute_force():
    """The definition, voxel by voxel, on a tiny volume (window clipped at the
    faces)."""
    x = synth.random_volume(5, 40)
    ss, sr, r = 0.9, 0.3, 1
    got = O.bilateral_filter(x, ss, sr, r)
    for p in [(0, 0, 0), (2, 3, 1), (4, 4, 4), (1, 0, 3)]:
        num = den = 0.0
        for q in np.ndindex(5, 5, 5):
            d = np.subtract(q, p)
            if np.abs(d).max() > r:
                continue
            w = math.exp(-float(d @ d) / (2 * ss * ss)) * math.exp(-(x[p] - x[q]) ** 2 / (2 * sr * sr))
            num += w * x[q]
            den += w
        assert math.isclose(got[p], num / den, rel_tol=1e-13)


def test_bilateral_limits():
    """A huge range sigma leaves the normalised Gaussian: in the interior it is
    scipy's correlation with the normalised kernel; a tiny one leaves the
    identity (no two random values are equal); constants are kept."""
    x = synth.random_volume(12, 41)
    g = np.array([[[math.exp(-((a - 2) ** 2 + (b - 2) ** 2 + (c - 2) ** 2) / (2 * 1.3 ** 2)) for c in range(5)]
                   for b in range(5)] for a in range(5)])
    g /= g.sum()
    wide = O.bilateral_filter(x, 1.3, 1e9, 2)
    ref = scipy.ndimage.correlate(x, g, mode="constant")
    np.testing.assert_allclose(wide[2:-2, 2:-2, 2:-2], ref[2:-2, 2:-2, 2:-2], rtol=0, atol=1e-12)
    np.testing.assert_allclose(O.bilateral_filter(x, 1.0, 1e-6, 1), x, rtol=0, atol=1e-12)
    c = np.full((6, 6, 6), 0.37)
    np.testing.assert_allclose(O.bilateral_filter(c, 1.0, 0.1, 2), c, rtol=1e-14)


def test_multigrid_bilateral_is_applied_after_each_landweber_step():
    """Alg. 1 order at one grid: Landweber step (with its soft threshold), then
    the bilateral filter."""
    n = 8
    scan = make_scan(n, nviews=6, seed=14)
    g = O.level_geometry(scan, 0)
    b = O.project(g, synth.random_volume(n, 15))
    mu0 = 0.1 * synth.random_volume(n, 16)
    got = O.multigrid(scan, mu0, [b], levels=1, lam=0.01, bilateral=(1.0, 0.2, 1))
    lw, _ = O.landweber_step(g, mu0, b, lam=0.01)
    np.testing.assert_allclose(got, O.bilateral_filter(lw, 1.0, 0.2, 1), rtol=0, atol=1e-13)


def _fas_case(n=16, nviews=40, levels=2):
    scan = make_scan(n, nviews=nviews, seed=21)
    ph = synth.ellipsoids(6, 3, axis_lo=0.08, axis_hi=0.3)
    x = synth.voxelize_ellipsoids(ph, n, supersample=1).numpy().astype(np.float64)
    b = O.project(O.level_geometry(scan, 0), x)
    return scan, x, O.data_levels(b, levels)


@pytest.mark.parametrize("levels", [2, 3])
def test_multigrid_fas_exact_solution_is_fixed_point(levels):
    """With consistent data b = P x and mu = x, the FAS coarse data is
    R (b - P x) + P_c R x = P_c R x, which the coarse solver leaves at R x,
    and the fine residual is zero: x is a fixed point.  The plain recursion
    (coarse data R b != P_c R x) moves away from it -- the plateau that FAS
    removes."""
    scan, x, bl = _fas_case(levels=levels)
    fas = O.multigrid(scan, x, bl, levels, fas=True)
    plain = O.multigrid(scan, x, bl, levels, fas=False)
    assert np.abs(fas - x).max() <= 1e-12 * np.abs(x).max()
    assert np.abs(plain - x).max() >= 1e-2 * np.abs(x).max()


def test_multigrid_fas_first_iteration_from_zero_is_plain():
    """From mu = 0 the FAS coarse data R (b - P 0) + P_c 0 is R b: the first
    iteration is the plain one."""
    scan, x, bl = _fas_case(n=8, nviews=12)
    mu0 = np.zeros_like(x)
    np.testing.assert_allclose(O.multigrid(scan, mu0, bl, 2, fas=True), O.multigrid(scan, mu0, bl, 2),
                               rtol=0, atol=1e-14)


def test_multigrid_fas_converges_past_the_plain_plateau():
    """On consistent data the plain recursion stalls (its fixed point is not
    the solution) while FAS keeps converging: after 24 iterations its error is
    below half the plain one and still falling."""
    scan, x, bl = _fas_case()
    rng = float(x.max() - x.min())
    err = {}
    for fas in (False, True):
        mu = np.zeros_like(x)
        e = []
        for _ in range(24):
            mu = O.multigrid(scan, mu, bl, 2, fas=fas)
            e.append(np.sqrt(np.mean((mu - x) ** 2)) / rng)
        err[fas] = e
    assert err[True][-1] < 0.5 * err[False][-1], (err[True][-1], err[False][-1])
    assert all(a > b for a, b in zip(err[True][-6:], err[True][-5:]))


@pytest.mark.slow
def test_pmgl_beats_sirt_at_equal_cost():
    """Sec. 3 / Fig. 4: after 2 iterations preconditioned multigrid Landweber is
    closer to the truth than SIRT with the same number of fine-grid P/B calls."""
    n = 32
    th, z = synth.trajectory(48, 2104)
    nu = 48
    scan = O.Scan(n=n, nu=nu, nv=nu, theta=th, z=z, pitch=synth.default_pitch(nu))
    ph = synth.ellipsoids(10, 2103)
    truth = synth.voxelize_ellipsoids(ph, n, supersample=2).numpy()
    b = O.ellipsoid_line_integrals(O.level_geometry(scan, 0), ph)
    mg = O.reconstruct(scan, b, iters=2, levels=2)
    sirt = O.sirt(scan, b, iters=2)
    e_mg = np.sqrt(np.mean((mg - truth) ** 2))
    e_sirt = np.sqrt(np.mean((sirt - truth) ** 2))
    assert e_mg < e_sirt, (e_mg, e_sirt)


# ---------------------------------------------------------------- geometry gradient

def _grad_scan(drift, n=20, nu=30, nviews=4):
    th, z = synth.trajectory(nviews, 3)
    return O.Scan(n=n, nu=nu, nv=nu, theta=th, z=0.3 * z, pitch=synth.default_pitch(nu), drift=drift)


def test_geometry_grad_matches_central_differences():
    """The analytic end-point derivative chained to phi equals central
    differences of the oracle's own P (step 1e-6 px: below the spacing of the
    bilinear interpolant's kinks, so the integral is locally smooth)."""
    K = 4
    drift = synth.drift_walk(K, 4, sigma_px=0.5, half_diag_px=20)
    ph = synth.blobs(3, 5, 0.08, 0.12, centre_r=0.15)
    vol = synth.voxelize_blobs(ph, 20).numpy()
    y = np.random.default_rng(0).standard_normal((K, 30, 30))
    gr = O.geometry_grad(_grad_scan(drift), vol, y)
    for k in range(K):
        for j in range(5):
            e = 1e-6 if j < 4 else 4e-8
            d1, d2 = drift.copy(), drift.copy()
            d1[k, j] += e
            d2[k, j] -= e
            a1 = O.project(O.level_geometry(_grad_scan(d1), 0), vol)[k]
            a2 = O.project(O.level_geometry(_grad_scan(d2), 0), vol)[k]
            fd = np.sum(y[k] * (a1 - a2)) / (2 * e)
            assert abs(gr[k, j] - fd) <= 1e-6 * max(abs(fd), np.abs(gr).max()), (k, j, gr[k, j], fd)


def test_geometry_grad_against_closed_form_blob():
    """Independent of Joseph: the drift derivative of the closed-form Gaussian
    line integral (central differences of the exact integral) against the
    oracle's gradient on the sampled blob; agreement to the discretisation
    error (measured 4.8 %, 2.2 %, 0.3 % of the largest entry at n = 20, 40, 80)."""
    K = 3
    drift = np.zeros((K, 5))
    drift[:, 4] = 0.02
    ph = synth.blobs(1, 9, 0.1, 0.1, centre_r=0.1)
    n = 48
    vol = synth.voxelize_blobs(ph, n).numpy()
    scan = _grad_scan(drift, n=n, nu=60, nviews=K)
    # weights = a ramp across the detector, so the derivatives are first
    # moments of the projection (a constant weight would nearly cancel them)
    uc = np.arange(60) - 29.5
    y = np.broadcast_to(1.0 + 0.05 * uc[None, None, :] + 0.03 * uc[None, :, None], (K, 60, 60)).copy()
    gr = O.geometry_grad(scan, vol, y)
    for j in range(5):
        e = 1e-4 if j < 4 else 4e-6
        d1, d2 = drift.copy(), drift.copy()
        d1[:, j] += e
        d2[:, j] -= e
        s1 = _grad_scan(d1, n=n, nu=60, nviews=K)
        s2 = _grad_scan(d2, n=n, nu=60, nviews=K)
        fd = (np.sum(y * O.blob_line_integrals(O.level_geometry(s1, 0), ph), axis=(1, 2))
              - np.sum(y * O.blob_line_integrals(O.level_geometry(s2, 0), ph), axis=(1, 2))) / (2 * e)
        scale = max(np.abs(fd).max(), 1e-3 * np.abs(gr).max())
        assert np.abs(gr[:, j] - fd).max() <= 0.03 * scale, (j, gr[:, j], fd)
