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
