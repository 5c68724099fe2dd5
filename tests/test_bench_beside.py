"""Host logic of the oracle-beside-GPU timings in bench.py: the A and A^T
voxel-view counts that extrapolate the oracle's solve time from its
per-operation rates must be those the oracle's two-iteration multigrid solve
actually makes (counted by wrapping its A and A^T), and the per-ray and
per-voxel-view rates must be finite and positive."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle as O  # noqa: E402
from paper_2103_10329_gb300 import synth  # noqa: E402


def _scan(n, nu, k):
    th, z = synth.trajectory(k, 7)
    return O.Scan(n=n, nu=nu, nv=nu, theta=th, z=z, pitch=synth.default_pitch(nu))


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_solve_units_match_the_oracle_calls(levels, monkeypatch):
    n, nu, k = 16, 20, 9
    scan = _scan(n, nu, k)
    counts = {"A": 0, "AT": 0}
    proj, back = O.project, O.backproject

    def cp(g, vol):
        counts["A"] += g.n ** 3 * g.n_views
        return proj(g, vol)

    def cb(g, sino):
        counts["AT"] += g.n ** 3 * g.n_views
        return back(g, sino)

    monkeypatch.setattr(O, "project", cp)
    monkeypatch.setattr(O, "backproject", cb)
    b = np.random.default_rng(1).random((k, nu, nu))
    O.reconstruct(scan, b, iters=2, levels=levels)
    assert bench._oracle_solve_units(n, k, levels) == (counts["A"], counts["AT"])


def test_ray_voxel_rates_positive():
    scan = _scan(16, 20, 9)
    og = O.level_geometry(scan, 0)
    vol = synth.random_volume(16, 2)
    t_ray, t_vox = bench._ray_voxel_rates(og, vol, 200, sino_views=3)
    assert np.isfinite(t_ray) and t_ray > 0
    assert np.isfinite(t_vox) and t_vox > 0


def test_count_nnz_matches_the_oracle_matrix():
    """The roofline's work count: bench.count_nnz counts, per ray, the major-
    axis planes whose sample lies within one voxel of the volume (so at least
    one bilinear tap is nonzero), times 4 taps.  At 8^3 the planes must be
    exactly those that hold a nonzero entry of the oracle's A, assembled
    column by column from A e_j."""
    n, nu, k = 8, 12, 3
    scan = _scan(n, nu, k)
    g = O.level_geometry(scan, 0)
    cols = []
    for j in range(n ** 3):
        e = np.zeros(n ** 3)
        e[j] = 1.0
        cols.append(O.project(g, e.reshape(n, n, n)).ravel())
    a = np.stack(cols, axis=1)  # rays x voxels, voxel j = (iz * n + iy) * n + ix
    iz, iy, ix = np.unravel_index(np.arange(n ** 3), (n, n, n))
    planes = 0
    for r in range(a.shape[0]):
        kv, ju = divmod(r, nu)
        kk, jv = divmod(kv, nu)
        w = g.det[kk] + ju * g.pu[kk] + jv * g.pv[kk] - g.src[kk]
        coord = iy if abs(w[1]) > abs(w[0]) else ix
        planes += len(np.unique(coord[a[r] != 0.0]))
    got = bench.count_nnz(scan.theta, scan.z, scan.pitch, n, nu, nu, device="cpu")
    assert planes > k * nu * nu  # most rays cross several planes
    assert got == 4.0 * planes
