"""Mixed-precision form: the projector and back-projector read 16-bit copies
(a BF16 or FP16 shadow of mu and of the search direction, a 16-bit residual
sinogram) while mu, b, the Eq. 5 filter and the update stay float32,
accumulation is float32, and the step size and norms float64.  The error of
each multigrid iterate against the FP64 oracle is reported and bounded.

Tolerance, from the arithmetic: every value the operators read carries a
relative storage rounding of at most u = 2^-9 (BF16) or 2^-11 (FP16); one
step reads two such copies (the shadow of mu through A, the residual through
A^T), so the update direction differs by O(2u) relative.  The bound on the
reconstruction difference is 2u of the phantom's range."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2103_10329_gb300 import synth
from tests.helpers import cuda, gpu_geom, oracle_scan, scan_desc, to_np

pytestmark = pytest.mark.gpu

U = {torch.bfloat16: 2.0 ** -9, torch.float16: 2.0 ** -11}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2103_10329_gb300 import build
    build.build()
    O.build()


@pytest.mark.parametrize("storage", [torch.bfloat16, torch.float16], ids=["bf16", "fp16"])
def test_multigrid_iterates_vs_fp64_oracle(storage):
    from paper_2103_10329_gb300 import mgct
    d = scan_desc(64, 96, 96, 90, 2104, levels=2)
    scan = oracle_scan(d)
    og = O.level_geometry(scan, 0)
    ph = synth.ellipsoids(10, 2103)
    truth = synth.voxelize_ellipsoids(ph, 64, supersample=2).numpy()
    b = O.ellipsoid_line_integrals(og, ph)
    rng = truth.max() - truth.min()
    bl = O.data_levels(b, 2)
    g = gpu_geom(d)
    rec = mgct.Reconstructor(g)
    rec.prepare(cuda(b))
    mu_o = np.zeros((64,) * 3)
    v32 = torch.zeros((64,) * 3, device="cuda")
    v16 = torch.zeros((64,) * 3, device="cuda")
    report = []
    for it in range(2):
        mu_o = O.multigrid(scan, mu_o, bl, levels=2)
        rec.iterate(v32)
        rec.iterate(v16, storage=storage)
        e32 = np.sqrt(np.mean((to_np(v32) - mu_o) ** 2)) / rng
        e16 = np.sqrt(np.mean((to_np(v16) - mu_o) ** 2)) / rng
        report.append((it + 1, e32, e16))
        assert e32 <= 1e-4, report
        assert e16 <= 2 * U[storage], report
    # and the 16-bit form still converges like the float32 one
    err16 = np.sqrt(np.mean((to_np(v16) - truth) ** 2))
    err32 = np.sqrt(np.mean((to_np(v32) - truth) ** 2))
    assert err16 <= err32 * (1 + 4 * U[storage]) + 2 * U[storage] * rng, (err16, err32)
    print(f"\n{storage}: iterate, RMSE(fp32 - oracle)/range, RMSE(16-bit - oracle)/range: {report}")


@pytest.mark.parametrize("storage", [torch.bfloat16, torch.float16], ids=["bf16", "fp16"])
def test_landweber_step_16bit_matches_fp32_within_storage_rounding(storage):
    from paper_2103_10329_gb300 import mgct
    d = scan_desc(48, 72, 72, 40, 2104, levels=1)
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    ph = synth.ellipsoids(10, 2103)
    b = cuda(O.ellipsoid_line_integrals(og, ph))
    mu0 = cuda(0.4 * synth.voxelize_ellipsoids(ph, 48, supersample=2).numpy())
    v32, v16 = mu0.clone(), mu0.clone()
    s32 = torch.zeros(4, dtype=torch.float64, device="cuda")
    s16 = torch.zeros(4, dtype=torch.float64, device="cuda")
    mgct.landweber_step(g, v32, b, stats=s32)
    mgct.landweber_step(g, v16, b, stats=s16, storage=storage)
    step32 = to_np(v32 - mu0)
    step16 = to_np(v16 - mu0)
    rel = np.linalg.norm(step16 - step32) / np.linalg.norm(step32)
    assert rel <= 4 * U[storage], rel
    # |r|^2 is computed from float32 residuals before the 16-bit store
    assert abs(s16[1].item() - s32[1].item()) <= 4 * U[storage] * s32[1].item()


def test_c3_mixed_precision_at_size():
    """The mixed-precision workload at its own size: 512^3 volume, 768^2
    detector, 1440 views, 3 grids, two multigrid iterations from zero in
    float32, BF16 and FP16 on the same data.  Per iteration and 16-bit form:

    (a) RMSE(16-bit iterate - float32 iterate) / range <= 2u, the storage
        rounding bound of the module docstring (the float32 iterate is the
        one the oracle checks at the smaller sizes);
    (b) the operators on the copies that form reads, against the FP64
        oracle on exactly those 16-bit values: A of the 16-bit shadow of mu
        at 300 sampled rays, and A^T of the residual rounded to 16 bits at
        24 sampled voxels (relative to A^T |y|), within the float32
        tolerance.  The oracle's voxel sums take the whole float64 sinogram
        on the host (6.8 GB)."""
    from paper_2103_10329_gb300 import mgct
    from tests.helpers import TOL_F32, check_err
    n, nu, K = 512, 768, 1440
    d = scan_desc(n, nu, nu, K, 2104, levels=3)
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    ph = synth.ellipsoids(50, 2103)
    truth = synth.voxelize_ellipsoids(ph, n, supersample=1, device="cuda", dtype=torch.float32)
    rng = float(truth.max() - truth.min())
    b = mgct.project(g, truth)
    del truth
    rec = mgct.Reconstructor(g)
    rec.prepare(b)
    forms = {"fp32": torch.float32, "bf16": torch.bfloat16, "fp16": torch.float16}
    vols = {k: torch.zeros((n, n, n), device="cuda") for k in forms}
    rays = synth.random_indices(300, (K, nu, nu), 31)
    ri = torch.as_tensor(rays, device="cuda", dtype=torch.long)
    vox = synth.random_indices(24, (n, n, n), 32)
    vi = torch.as_tensor(vox, device="cuda", dtype=torch.long)
    report = []
    for it in range(2):
        for name, st in forms.items():
            rec.iterate(vols[name], storage=st)
        torch.cuda.synchronize()
        for name in ("bf16", "fp16"):
            st = forms[name]
            u = U[st]
            diff = float(torch.sqrt(torch.mean((vols[name].double() - vols["fp32"].double()) ** 2))) / rng
            # (b) A of the shadow this form reads
            shadow = vols[name].to(st)
            proj = mgct.project(g, shadow)
            sh_np = to_np(shadow)
            ref = O.project_rays(og, sh_np, rays)
            got = to_np(proj[ri[:, 0], ri[:, 1], ri[:, 2]])
            ea = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-2 * float(proj.abs().max()))
            # (b) A^T of the 16-bit residual
            r16 = (b - mgct.project(g, vols[name])).to(st)
            del proj, shadow, sh_np
            bp = mgct.backproject(g, r16)
            r_np = to_np(r16)
            del r16
            refv = O.backproject_voxels(og, r_np, vox, radius=5)
            absv = O.backproject_voxels(og, np.abs(r_np), vox, radius=5)
            del r_np
            gotv = to_np(bp[vi[:, 2], vi[:, 1], vi[:, 0]])
            del bp
            ev = np.abs(gotv - refv) / np.maximum(absv, 1e-2 * absv.max())
            report.append({"iter": it + 1, "form": name, "rmse_vs_fp32_over_range": diff,
                           "A_max_rel": float(ea.max()), "AT_max_rel": float(ev.max())})
            assert diff <= 2 * u, report
            check_err(ea, TOL_F32)
            check_err(ev, TOL_F32)
            torch.cuda.empty_cache()
    print("\nc3 mixed precision per iteration:", report)
