"""GPU parity of the operators (A, A^T, p, R, P) against the FP64 oracle,
called through the C ABI."""
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


C1 = dict(n=64, nu=96, nv=96, nviews=90, seed=2104, levels=2)


def c1_desc(**kw):
    d = dict(C1)
    d.update(kw)
    return scan_desc(d["n"], d["nu"], d["nv"], d["nviews"], d["seed"], levels=d["levels"],
                     drift=d.get("drift"))


def drift_desc(n=24, nu=36, nv=20, nviews=7, seed=31):
    drift = synth.drift_walk(nviews, seed + 1, sigma_px=2.0, half_diag_px=0.5 * np.hypot(nu, nv))
    return scan_desc(n, nu, nv, nviews, seed, levels=1, drift=drift)


from paper_2103_10329_gb300 import mgct  # noqa: E402


# --------------------------------------------------------------------------- A

@pytest.mark.parametrize("which", ["random", "phantom"])
def test_project_c1(which):
    d = c1_desc()
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    if which == "random":
        vol = synth.random_volume(64, 5)
    else:
        vol = synth.voxelize_ellipsoids(synth.ellipsoids(10, 2103), 64, supersample=2).numpy()
    vol32 = vol.astype(np.float32)
    ref = O.project(og, vol32.astype(np.float64))
    got = to_np(mgct.project(g, cuda(vol32)))
    e = rel_err(got, ref)
    check_err(e, TOL_F32)


def test_project_ragged_drift_tilt():
    """Ragged tiles (n=24, 36x20 detector, 7 views) with source/detector
    drift and detector tilt."""
    d = drift_desc()
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    vol = synth.random_volume(24, 6).astype(np.float32)
    ref = O.project(og, vol.astype(np.float64))
    got = to_np(mgct.project(g, cuda(vol)))
    e = rel_err(got, ref)
    check_err(e, TOL_F32)


def test_project_coarse_level_and_view_subset():
    d = c1_desc()
    g = gpu_geom(d)
    og1 = O.level_geometry(oracle_scan(d), 1)
    vol = synth.random_volume(32, 7).astype(np.float32)
    views = np.arange(3, 90, 8)
    ref = O.project(og1.subset(views), vol.astype(np.float64))
    got = to_np(mgct.project(g, cuda(vol), level=1, views=(3, len(views), 8)))
    e = rel_err(got, ref)
    check_err(e, TOL_F32)


def test_project_residual_and_norm():
    d = c1_desc()
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    vol = synth.random_volume(64, 8).astype(np.float32)
    b = (O.project(og, vol.astype(np.float64)) * 1.01 + 0.001).astype(np.float32)
    ss = torch.zeros(1, dtype=torch.float64, device="cuda")
    r = to_np(mgct.project(g, cuda(vol), b=cuda(b), sumsq=ss))
    ref = b.astype(np.float64) - O.project(og, vol.astype(np.float64))
    assert np.abs(r - ref).max() <= 2e-5 * np.abs(b).max()
    assert abs(ss.item() - np.sum(r * r)) <= 1e-9 * np.sum(r * r)


@pytest.mark.parametrize("vt,ot", [(torch.bfloat16, torch.float32), (torch.float16, torch.float32),
                                   (torch.float32, torch.bfloat16), (torch.float32, torch.float16)])
def test_project_storage_dtypes(vt, ot):
    """Form 1: bf16/fp16 storage, float32 accumulation.  The oracle projects
    the rounded volume; the output error is the storage rounding of ot."""
    d = c1_desc(n=32, nu=48, nv=48, nviews=20)
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    vol = cuda(synth.random_volume(32, 9)).to(vt)
    ref = O.project(og, to_np(vol))
    got = to_np(mgct.project(g, vol, out_dtype=ot))
    e = rel_err(got, ref)
    tol = {torch.float32: TOL_F32, torch.bfloat16: 2 ** -8, torch.float16: 2 ** -11}[ot]
    check_err(e, tol)


def test_project_empty_selection():
    d = c1_desc(n=32, nu=48, nv=48, nviews=10)
    g = gpu_geom(d)
    out = mgct.project(g, torch.ones((32, 32, 32), device="cuda"), views=(0, 0, 1))
    assert out.shape == (0, 48, 48)
    torch.cuda.synchronize()


# --------------------------------------------------------------------------- A^T

@pytest.mark.parametrize("kind", ["uniform", "normal"])
def test_backproject_c1(kind):
    d = c1_desc()
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    rng = np.random.default_rng(11)
    y = rng.random((90, 96, 96)) if kind == "uniform" else rng.standard_normal((90, 96, 96))
    y32 = y.astype(np.float32)
    ref = O.backproject(og, y32.astype(np.float64))
    got = to_np(mgct.backproject(g, cuda(y32)))
    # signed data: the error of a sum is measured against the sum of the
    # magnitudes of its terms, A^T |y| (equal to |A^T y| for y >= 0)
    scale = O.backproject(og, np.abs(y32.astype(np.float64)))
    e = rel_err(got, ref) if kind == "uniform" else np.abs(got - ref) / np.maximum(scale, 1e-2 * scale.max())
    check_err(e, TOL_F32)


def test_backproject_ragged_drift_tilt_and_accumulate():
    """The general (tilted) gather against the oracle; accumulate adds the
    same float32 sums to the output, one rounding each, as torch's add."""
    d = drift_desc()
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    y = np.random.default_rng(12).random((7, 20, 36)).astype(np.float32)
    ref = O.backproject(og, y.astype(np.float64))
    plain = mgct.backproject(g, cuda(y))
    check_err(rel_err(to_np(plain), ref), TOL_F32)
    out = torch.full((24, 24, 24), 0.5, device="cuda")
    got = mgct.backproject(g, cuda(y), out=out, accumulate=True)
    assert torch.equal(got, plain + 0.5)


def test_backproject_subset_and_storage_dtypes():
    d = c1_desc(n=32, nu=48, nv=48, nviews=24)
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    views = np.arange(2, 24, 5)
    y = cuda(np.random.default_rng(13).random((len(views), 48, 48))).to(torch.bfloat16)
    ref = O.backproject(og.subset(views), to_np(y))
    got = to_np(mgct.backproject(g, y, views=(2, len(views), 5)))
    e = rel_err(got, ref)
    check_err(e, TOL_F32)
    y16 = y.to(torch.float16)
    got16 = to_np(mgct.backproject(g, y16, views=(2, len(views), 5)))
    e16 = rel_err(got16, O.backproject(og.subset(views), to_np(y16)))
    check_err(e16, TOL_F32)


@pytest.mark.parametrize("case", ["chunked", "scratch_too_small"])
def test_backproject_chunks_and_fallback(case):
    """The public A^T weights the caller's rays into the quad scratch,
    8 (n+5)^2 n floats, and splats them with the slab kernel.  At n = 16 with
    a 48^2 detector the scratch holds 24 views, so 60 views run as chunks of
    24, 24 and 12 (the later ones accumulating); at n = 8 with a 112^2
    detector it holds less than one view and the call takes the per-voxel
    gather instead.  Both against the oracle, plain and accumulating."""
    n, nu, k = (16, 48, 60) if case == "chunked" else (8, 112, 6)
    d = scan_desc(n, nu, nu, k, 41, levels=1)
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    y = np.random.default_rng(42).random((k, nu, nu)).astype(np.float32)
    ref = O.backproject(og, y.astype(np.float64))
    got = to_np(mgct.backproject(g, cuda(y)))
    e = rel_err(got, ref)
    check_err(e, TOL_F32)
    out = torch.full((n, n, n), 0.5, device="cuda")
    got = to_np(mgct.backproject(g, cuda(y), out=out, accumulate=True)) - 0.5
    e = rel_err(got, ref)
    check_err(e, 2 * TOL_F32)


def test_backproject_empty_selection_gives_zero():
    d = c1_desc(n=32, nu=48, nv=48, nviews=10)
    g = gpu_geom(d)
    out = torch.full((32, 32, 32), 3.0, device="cuda")
    mgct.backproject(g, torch.empty((0, 48, 48), device="cuda"), views=(0, 0, 1), out=out)
    assert float(out.abs().max()) == 0.0


def test_gpu_adjoint_identity():
    """Sec. 2.1: B is the adjoint of P.  Both GPU kernels share the ray
    set-up, so <A x, y> = <x, A^T y> up to float32 summation error."""
    d = c1_desc()
    g = gpu_geom(d)
    x = cuda(synth.random_volume(64, 14))
    y = cuda(np.random.default_rng(15).standard_normal((90, 96, 96)))
    ax = mgct.project(g, x)
    aty = mgct.backproject(g, y)
    lhs = float(torch.sum(ax.double() * y.double()))
    rhs = float(torch.sum(x.double() * aty.double()))
    scale = float(torch.sum(ax.double().abs() * y.double().abs()))
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_determinism():
    d = c1_desc()
    g = gpu_geom(d)
    x = cuda(synth.random_volume(64, 16))
    y = cuda(np.random.default_rng(17).standard_normal((90, 96, 96)))
    a1, a2 = mgct.project(g, x), mgct.project(g, x)
    b1, b2 = mgct.backproject(g, y), mgct.backproject(g, y)
    assert torch.equal(a1, a2) and torch.equal(b1, b2)


# --------------------------------------------------------------------------- full-size samples

@pytest.mark.parametrize("cfg", [(256, 384, 720), (512, 768, 1440), (1024, 1536, 2880)], ids=["c2", "c3", "c5"])
def test_full_size_sampled(cfg):
    """At the benchmark sizes (and the 1024^3 / 1536^2 / 2880-view evaluation
    size of the learned form), in the launch configuration the bench times:
    sampled rays and voxels against the oracle computed one by one.  A runs
    over every view; at 1024^3 A^T runs over every 40th view (the oracle's
    voxel sums take the whole float64 sinogram on the host)."""
    n, nu, nviews = cfg
    d = scan_desc(n, nu, nu, nviews, 2104, levels=1)
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    ph = synth.ellipsoids(40, 2103, axis_lo=0.02, axis_hi=0.12)
    vol = synth.voxelize_ellipsoids(ph, n, supersample=1, device="cuda", dtype=torch.float32)
    proj = mgct.project(g, vol)
    rays = synth.random_indices(300, (nviews, nu, nu), 3)
    vol_np = to_np(vol)
    ref = O.project_rays(og, vol_np, rays)
    ri = torch.as_tensor(rays, device="cuda", dtype=torch.long)
    got = to_np(proj[ri[:, 0], ri[:, 1], ri[:, 2]])
    full_max = float(proj.abs().max())
    e = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-2 * full_max)
    check_err(e, TOL_F32)
    del vol, proj, vol_np
    stride = 40 if n >= 1024 else 1
    views = (0, len(range(0, nviews, stride)), stride)
    y = torch.rand((views[1], nu, nu), device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    bp = mgct.backproject(g, y, views=views)
    vox = synth.random_indices(24, (n, n, n), 5)
    sub = np.arange(0, nviews, stride)
    og_s = O.level_geometry(oracle_scan(dict(d, theta=d["theta"][sub], z=d["z"][sub])), 0)
    refv = O.backproject_voxels(og_s, to_np(y), vox, radius=5)
    vi = torch.as_tensor(vox, device="cuda", dtype=torch.long)
    gotv = to_np(bp[vi[:, 2], vi[:, 1], vi[:, 0]])
    ev = np.abs(gotv - refv) / np.maximum(np.abs(refv), 1e-2 * float(bp.abs().max()))
    check_err(ev, TOL_F32)


# --------------------------------------------------------------------------- p, R, P

@pytest.mark.parametrize("axis,n", [(2, 40), (2, 37), (2, 150), (0, 40), (1, 33)])
def test_precondition(axis, n):
    """Eq. 5 against the oracle: the z-slice stream kernel (vector and scalar
    staging, partial tiles) and the generic stencil for the other axes."""
    d = scan_desc(n, 48, 48, 4, 1, levels=1, slice_axis=axis)
    g = gpu_geom(d)
    x = synth.random_volume(n, 18).astype(np.float32) - 0.5
    ref = O.precondition(x.astype(np.float64), axis)
    got = to_np(mgct.precondition(g, cuda(x)))
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(x).max()


def test_restrict_and_prolong():
    x = synth.random_volume(48, 19).astype(np.float32)
    got = to_np(mgct.restrict_volume(cuda(x)))
    assert np.abs(got - O.restrict_volume(x.astype(np.float64))).max() <= 1e-6
    b = np.random.default_rng(20).random((5, 36, 52)).astype(np.float32)
    got = to_np(mgct.restrict_sino(cuda(b)))
    assert np.abs(got - O.restrict_sino(b.astype(np.float64))).max() <= 1e-6
    for nc in (20, 131):  # one and two 128-wide blocks along x
        cn = synth.random_volume(nc, 21).astype(np.float32)
        co = synth.random_volume(nc, 22).astype(np.float32)
        fine = synth.random_volume(2 * nc, 23).astype(np.float32)
        ref = fine.astype(np.float64) + O.prolong(cn.astype(np.float64) - co.astype(np.float64))
        got = to_np(mgct.prolong_add(cuda(cn), cuda(co), cuda(fine)))
        assert np.abs(got - ref).max() <= 1e-6


@pytest.mark.parametrize("n,nu,nv,nviews", [(48, 72, 72, 30), (37, 55, 41, 11), (40, 40, 40, 12), (24, 72, 72, 8)],
                         ids=["rows-finer", "ragged", "rows-coarser", "rows-3x-finer"])
def test_solver_backprojection_detector_ratios(n, nu, nv, nviews):
    """The solver's A^T against the oracle at every voxel, for detectors whose
    rows step the crossing height by 1/3 < E1 < 1 voxel at every plane the
    rays cross (the register kernel: the first two cases, the second with
    ragged tiles) and for detectors outside that range (the shared-memory
    slab kernel): E1 above 1 at the far planes (n = nu) and below 1/3 at the
    near ones (nu = 3n).  With this scan's pitch the step at the volume
    centre is about 1.03 n / nu, and it varies by about -35 % / +35 % from
    the nearest to the farthest plane."""
    d = scan_desc(n, nu, nv, nviews, 2104, levels=1)
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    y = np.random.default_rng(8).random((nviews, nv, nu)).astype(np.float32)
    stats = torch.zeros(4, dtype=torch.float64, device="cuda")
    step = mgct.landweber_direction(g, torch.zeros((n, n, n), device="cuda"), cuda(y), precond=False, stats=stats)
    alpha = float(stats[0])
    assert alpha > 0
    got = to_np(step) / alpha
    ref = O.backproject(og, y.astype(np.float64))
    e = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-2 * np.abs(ref).max())
    check_err(e, TOL_F32)


@pytest.mark.parametrize("cfg", [(256, 384, 720), (512, 768, 1440)], ids=["c2", "c3"])
def test_solver_backprojection_full_size_sampled(cfg):
    """The solver's own A^T (the dl-weighted residual written by the
    projector's epilogue, then the register back-projector), in the launch
    configuration the bench times: with mu = 0 and no filter the Landweber
    direction is alpha A^T b, so A^T b = step / alpha; sampled voxels
    against the oracle."""
    n, nu, nviews = cfg
    d = scan_desc(n, nu, nu, nviews, 2104, levels=1)
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    y = torch.rand((nviews, nu, nu), device="cuda", generator=torch.Generator("cuda").manual_seed(6))
    stats = torch.zeros(4, dtype=torch.float64, device="cuda")
    step = mgct.landweber_direction(g, torch.zeros((n, n, n), device="cuda"), y, precond=False, stats=stats)
    alpha = float(stats[0])
    assert alpha > 0
    vox = synth.random_indices(24, (n, n, n), 7)
    vi = torch.as_tensor(vox, device="cuda", dtype=torch.long)
    got = to_np(step[vi[:, 2], vi[:, 1], vi[:, 0]]) / alpha
    ref = O.backproject_voxels(og, to_np(y), vox, radius=5)
    e = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-2 * float(step.abs().max()) / alpha)
    check_err(e, TOL_F32)
