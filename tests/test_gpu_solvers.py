"""GPU parity of the solvers (Landweber / SIRT step, OS-EMTR pass, the
multigrid iteration of Alg. 1) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2103_10329_gb300 import synth
from tests.helpers import check_err, cuda, gpu_geom, oracle_scan, scan_desc, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2103_10329_gb300 import build
    build.build()
    O.build()


from paper_2103_10329_gb300 import mgct  # noqa: E402


def phantom(n, seed=2103, count=10):
    ph = synth.ellipsoids(count, seed)
    return ph, synth.voxelize_ellipsoids(ph, n, supersample=2).numpy()


@pytest.mark.parametrize("precond,alpha,lam", [(True, None, 0.0), (False, None, 0.0),
                                               (True, 0.5, 0.0), (True, None, 1e-3)])
def test_landweber_step(precond, alpha, lam):
    d = scan_desc(48, 72, 72, 40, 2104, levels=1)
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    ph, truth = phantom(48)
    b = O.ellipsoid_line_integrals(og, ph).astype(np.float32)
    mu0 = (0.5 * truth).astype(np.float32)
    ref, st = O.landweber_step(og, mu0.astype(np.float64), b.astype(np.float64), alpha=alpha, lam=lam,
                               precond=precond)
    vol = cuda(mu0)
    stats = torch.zeros(4, dtype=torch.float64, device="cuda")
    mgct.landweber_step(g, vol, cuda(b), alpha=alpha, lam=lam, precond=precond, stats=stats)
    s = stats.cpu().numpy()
    assert abs(s[0] - st["alpha"]) <= 1e-4 * abs(st["alpha"])
    assert abs(s[1] - st["r2"]) <= 1e-5 * st["r2"]
    assert s[3] == 0.0
    check_err(np.abs(to_np(vol) - ref) / np.abs(ref).max(), 1e-5)


def test_osemtr_pass():
    d = scan_desc(32, 48, 48, 40, 2104, levels=1)
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    ph, truth = phantom(32)
    b = O.ellipsoid_line_integrals(og, ph).astype(np.float32)
    pi = O.project(og, np.ones((32, 32, 32)))
    mu0 = (0.8 * truth).astype(np.float32)
    ref = O.osemtr_pass(og, mu0.astype(np.float64), b.astype(np.float64), n_subsets=8, pi_sino=pi)
    vol = cuda(mu0)
    mgct.osemtr_pass(g, vol, cuda(b), cuda(pi), n_subsets=8)
    check_err(np.abs(to_np(vol) - ref) / np.abs(ref).max(), 1e-4)


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_multigrid_c1(levels):
    """Two iterations of Alg. 1 on the 64^3 / 96^2 / 90-view workload (analytic
    ellipsoid data): GPU vs oracle reconstruction RMSE difference <= 1e-4 of
    the phantom's range."""
    d = scan_desc(64, 96, 96, 90, 2104, levels=levels)
    scan = oracle_scan(d)
    og = O.level_geometry(scan, 0)
    ph, truth = phantom(64)
    b = O.ellipsoid_line_integrals(og, ph)
    ref = O.reconstruct(scan, b, iters=2, levels=levels)
    g = gpu_geom(d)
    rec = mgct.Reconstructor(g)
    rec.prepare(cuda(b))
    got = to_np(rec.reconstruct(iters=2))
    rng = truth.max() - truth.min()
    check_err(np.abs(got - ref) / rng, 1e-4, bound="rms")
    # and the method reconstructs: error well below the phantom's own RMS
    if levels > 1:
        assert np.sqrt(np.mean((got - truth) ** 2)) < 0.6 * np.sqrt(np.mean(truth ** 2))


@pytest.mark.parametrize("levels", [2, 3])
def test_multigrid_fas_c1(levels):
    """Three iterations of the FAS variant (coarse data R(b - A mu) + A_c R mu)
    on the 64^3 / 96^2 / 90-view workload: GPU vs oracle reconstruction RMSE
    difference <= 1e-4 of the phantom's range."""
    d = scan_desc(64, 96, 96, 90, 2104, levels=levels)
    scan = oracle_scan(d)
    og = O.level_geometry(scan, 0)
    ph, truth = phantom(64)
    b = O.ellipsoid_line_integrals(og, ph)
    ref = O.reconstruct(scan, b, iters=3, levels=levels, fas=True)
    g = gpu_geom(d)
    rec = mgct.Reconstructor(g)
    rec.prepare(cuda(b))
    got = to_np(rec.reconstruct(iters=3, fas=True))
    rng = truth.max() - truth.min()
    check_err(np.abs(got - ref) / rng, 1e-4, bound="rms")


def test_multigrid_fas_keeps_the_exact_solution():
    """Consistent data b = A x (oracle) and mu = x: one FAS iteration leaves mu
    at x up to float32 rounding; the plain recursion moves it by percents."""
    d = scan_desc(32, 48, 48, 40, 2104, levels=2)
    scan = oracle_scan(d)
    _, x = phantom(32)
    b = cuda(O.project(O.level_geometry(scan, 0), x.astype(np.float64)))
    g = gpu_geom(d)
    rec = mgct.Reconstructor(g)
    rec.prepare(b)
    moved = {}
    for fas in (True, False):
        v = cuda(x).clone()
        rec.iterate(v, fas=fas)
        moved[fas] = float((v - cuda(x)).abs().max()) / float(np.abs(x).max())
    assert moved[True] <= 1e-4, moved
    assert moved[False] >= 1e-2, moved


@pytest.mark.parametrize("n,ss,sr,r", [(24, 1.0, 0.2, 1), (37, 1.5, 0.05, 2), (20, 2.0, 1.0, 3)])
def test_bilateral_filter(n, ss, sr, r):
    """Alg. 1 BilateralFilter against the oracle (clipped window at the faces,
    an odd size, radii 1-3); float32 with __expf weights: 1e-5 of the range."""
    x = synth.random_volume(n, 50 + r).astype(np.float32)
    ref = O.bilateral_filter(x.astype(np.float64), ss, sr, r)
    got = to_np(mgct.bilateral(cuda(x), ss, sr, r))
    assert np.abs(got - ref).max() <= 1e-5 * (x.max() - x.min())


def test_multigrid_with_bilateral_c1():
    """Two iterations of Alg. 1 with the BilateralFilter after every grid's
    Landweber step, on the 64^3 / 96^2 / 90-view workload, 2 grids: GPU vs
    oracle reconstruction RMSE difference <= 1e-4 of the phantom's range."""
    d = scan_desc(64, 96, 96, 90, 2104, levels=2)
    scan = oracle_scan(d)
    og = O.level_geometry(scan, 0)
    ph, truth = phantom(64)
    b = O.ellipsoid_line_integrals(og, ph)
    bil = (1.0, 0.1, 1)
    ref = O.reconstruct(scan, b, iters=2, levels=2, bilateral=bil)
    g = gpu_geom(d)
    rec = mgct.Reconstructor(g)
    rec.prepare(cuda(b))
    got = to_np(rec.reconstruct(iters=2, bilateral=bil))
    rng = truth.max() - truth.min()
    assert np.sqrt(np.mean((got - ref) ** 2)) / rng <= 1e-4
    plain = O.reconstruct(scan, b, iters=2, levels=2)
    assert np.abs(ref - plain).max() > 1e-3  # the filter did act


def test_custom_preconditioner_kernel():
    """A kernel set on the geometry replaces Eq. 5: mgct_precondition with an
    asymmetric kernel, and two multigrid iterations (2 grids), against the
    oracle with the same kernel."""
    k = np.random.default_rng(70).standard_normal((3, 3, 3))
    d = scan_desc(40, 48, 48, 4, 1, levels=1)
    g = gpu_geom(d)
    g.set_preconditioner(k)
    x = synth.random_volume(40, 71).astype(np.float32) - 0.5
    got = to_np(mgct.precondition(g, cuda(x)))
    ref = O.precondition(x.astype(np.float64), kernel=k.astype(np.float32).astype(np.float64))
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    g.set_preconditioner(None)
    assert np.abs(to_np(mgct.precondition(g, cuda(x))) - O.precondition(x.astype(np.float64))).max() <= 1e-6
    # in the solver
    kk = np.zeros((3, 3, 3))
    kk[1, 1, 1] = 1.0
    kk[1, 1, 0] = kk[1, 1, 2] = kk[1, 0, 1] = kk[1, 2, 1] = -0.12
    kk[0, 1, 1] = kk[2, 1, 1] = -0.05
    d = scan_desc(64, 96, 96, 90, 2104, levels=2)
    scan = oracle_scan(d)
    scan.p_kernel = kk.astype(np.float32).astype(np.float64)
    ph, truth = phantom(64)
    b = O.ellipsoid_line_integrals(O.level_geometry(scan, 0), ph)
    ref = O.reconstruct(scan, b, iters=2, levels=2)
    g = gpu_geom(d)
    g.set_preconditioner(kk)
    rec = mgct.Reconstructor(g)
    rec.prepare(cuda(b))
    got = to_np(rec.reconstruct(iters=2))
    assert np.sqrt(np.mean((got - ref) ** 2)) / (truth.max() - truth.min()) <= 1e-4


def test_bilateral_argument_checks():
    x = cuda(np.zeros((8, 8, 8), np.float32))
    for args in [(0.0, 0.1, 1), (1.0, 0.0, 1), (1.0, 0.1, 0), (1.0, 0.1, 5)]:
        with pytest.raises(mgct.MgctError):
            mgct.bilateral(x, *args)
    with pytest.raises(mgct.MgctError):
        mgct.bilateral(x, 1.0, 0.1, 1, out=x)


def test_multigrid_matches_explicit_steps():
    """The native Alg. 1 driver equals the same steps issued one by one
    through the C ABI (restrict, OS-EMTR, prolong-add, Landweber)."""
    d = scan_desc(32, 48, 48, 24, 2104, levels=2)
    scan = oracle_scan(d)
    og = O.level_geometry(scan, 0)
    ph, truth = phantom(32)
    b = cuda(O.ellipsoid_line_integrals(og, ph))
    g = gpu_geom(d)
    rec = mgct.Reconstructor(g)
    rec.prepare(b)
    v1 = torch.zeros((32, 32, 32), device="cuda")
    rec.iterate(v1)
    b1 = mgct.restrict_sino(b)
    pi = mgct.project(g, torch.ones((16, 16, 16), device="cuda"), level=1)
    v2 = torch.zeros((32, 32, 32), device="cuda")
    mc = mgct.restrict_volume(v2)
    old = mc.clone()
    mgct.osemtr_pass(g, mc, b1, pi, level=1, n_subsets=8)
    mgct.prolong_add(mc, old, v2)
    mgct.landweber_step(g, v2, b, level=0)
    assert torch.equal(v1, v2)


def test_multigrid_deterministic():
    d = scan_desc(32, 48, 48, 24, 2104, levels=2)
    og = O.level_geometry(oracle_scan(d), 0)
    ph, _ = phantom(32)
    b = cuda(O.ellipsoid_line_integrals(og, ph))
    outs = []
    for _ in range(2):
        g = gpu_geom(d)
        rec = mgct.Reconstructor(g)
        rec.prepare(b)
        outs.append(rec.reconstruct(iters=2))
    assert torch.equal(outs[0], outs[1])


def test_nonfinite_data_is_reported_and_leaves_mu_untouched():
    """Failure detection without a GPU fault: a NaN in the data makes the
    step size non-finite; the device stats flag it, alpha is replaced by 0
    and the estimate is left exactly as it was."""
    d = scan_desc(32, 48, 48, 12, 2104, levels=1)
    g = gpu_geom(d)
    og = O.level_geometry(oracle_scan(d), 0)
    ph, truth = phantom(32)
    b = O.ellipsoid_line_integrals(og, ph).astype(np.float32)
    b[3, 20, 20] = np.nan
    mu = cuda(0.5 * truth)
    before = mu.clone()
    stats = torch.zeros(4, dtype=torch.float64, device="cuda")
    mgct.landweber_step(g, mu, cuda(b), stats=stats)
    s = stats.cpu().numpy()
    assert s[3] == 1.0 and s[0] == 0.0
    assert torch.equal(mu, before)
    # clean data: no flag
    b[3, 20, 20] = 0.0
    mgct.landweber_step(g, mu, cuda(b), stats=stats)
    assert stats[3].item() == 0.0 and stats[0].item() > 0.0
