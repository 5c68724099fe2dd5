"""The seeded synthetic inputs follow the stated recipe: trajectory strata,
detector coverage of the inscribed cylinder, ellipsoid phantom statistics,
the porous texture's porosity and Poisson log data.  CPU only."""
import math

import numpy as np
import torch

import oracle as O
from paper_2103_10329_gb300 import synth


def test_trajectory_golden_angle_and_strata():
    k = 720
    th, z = synth.trajectory(k, 3)
    steps = np.mod(np.diff(th), 2 * np.pi)
    np.testing.assert_allclose(steps, 2 * np.pi * 0.618034, rtol=0, atol=1e-9)
    # one source height per stratum of the volume's height, increasing
    strata = np.floor((z + 0.5) * k)
    np.testing.assert_array_equal(strata, np.arange(k))
    assert np.all(np.diff(z) > 0)
    th2, z2 = synth.trajectory(k, 3)
    np.testing.assert_array_equal(z, z2)


def test_detector_covers_the_inscribed_cylinder():
    """The outermost pixel centres' rays pass the rotation axis at about the
    cylinder radius 1/2 (within the half pixel the centres leave out)."""
    nu = 96
    pitch = synth.default_pitch(nu)
    scan = O.Scan(n=64, nu=nu, nv=nu, theta=np.array([0.3]), z=np.array([0.0]), pitch=pitch)
    g = O.level_geometry(scan, 0)
    src = g.src[0]
    for ju in (0, nu - 1):
        p = g.det[0] + ju * g.pu[0] + (nu // 2) * g.pv[0]
        w = p - src
        # in-plane distance from the z axis to the line src + t w
        a = np.array([w[0], w[1]])
        s = np.array([src[0], src[1]])
        d = abs(s[0] * a[1] - s[1] * a[0]) / np.linalg.norm(a)
        half_px = 0.5 * pitch * 2.0 / 4.0  # half a pixel, scaled from the detector to the axis
        assert 0.5 - half_px - 1e-12 <= d <= 0.5 + 1e-12, d


def test_ellipsoid_statistics():
    ph = synth.ellipsoids(4000, 7, axis_lo=0.01, axis_hi=0.08)
    c = ph["centre"]
    r = np.hypot(c[:, 0], c[:, 1])
    assert r.max() <= 0.35 and np.abs(c[:, 2]).max() <= 0.35
    # uniform in the disc: the median radius is 0.35 / sqrt(2)
    assert abs(np.median(r) - 0.35 / math.sqrt(2)) < 0.01
    assert ph["axes"].min() >= 0.01 and ph["axes"].max() <= 0.08
    assert 0.0 <= ph["mu"].min() and ph["mu"].max() < 1.0
    rot = ph["rot"]
    eye = np.einsum("nij,nik->njk", rot, rot)
    np.testing.assert_allclose(eye, np.broadcast_to(np.eye(3), eye.shape), atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(rot), 1.0, atol=1e-12)


def test_porous_texture_porosity():
    """Pores where the normalised blurred noise exceeds 0.5: a fraction
    1 - Phi(0.5) = 0.309 of the solid cylinder, before the final blur."""
    n = 128
    tex = synth.porous_texture(n, 11, dtype=torch.float64).numpy()
    assert tex.min() >= -1e-12 and tex.max() <= 0.3 + 1e-9
    c = (np.arange(n) - (n - 1) / 2) / n
    r2 = c[None, :, None] ** 2 + c[None, None, :] ** 2
    core = (r2 <= 0.4 ** 2) & (np.abs(c)[:, None, None] <= 0.4)
    pore = tex[np.broadcast_to(core, tex.shape)] < 0.15
    assert abs(pore.mean() - (1 - 0.5 * (1 + math.erf(0.5 / math.sqrt(2))))) < 0.03
    outside = (r2 >= 0.5 ** 2) | (np.abs(c)[:, None, None] >= 0.5)
    assert np.abs(tex[np.broadcast_to(outside, tex.shape)]).max() < 1e-3


def test_poisson_log_data_is_unbiased_at_high_counts():
    b = torch.full((200000,), 1.0, dtype=torch.float64)
    y = synth.poisson_log_data(b, 1e4, 5).double()
    # -ln(I / I0) has mean b + Var(I) / (2 E[I]^2) + ... = b + 1 / (2 I0 e^-b)
    bias = 1.0 / (2 * 1e4 * math.exp(-1.0))
    assert abs(float(y.mean()) - (1.0 + bias)) < 3e-4
    # and standard deviation 1 / sqrt(I0 e^-b)
    assert abs(float(y.std()) - 1.0 / math.sqrt(1e4 * math.exp(-1.0))) < 5e-4


def test_poisson_log_data_in_view_blocks():
    """Sinograms larger than the block limit are drawn a block of whole views
    at a time: the same statistics, every view filled, and the single-draw
    result unchanged below the limit."""
    b = torch.full((50, 40, 100), 1.0, dtype=torch.float64)
    y = synth.poisson_log_data(b, 1e4, 5, chunk=7 * 4000 + 13).double()
    assert y.shape == b.shape and bool(torch.isfinite(y).all())
    bias = 1.0 / (2 * 1e4 * math.exp(-1.0))
    assert abs(float(y.mean()) - (1.0 + bias)) < 3e-4
    assert abs(float(y.std()) - 1.0 / math.sqrt(1e4 * math.exp(-1.0))) < 5e-4
    per_view = y.reshape(50, -1).std(dim=1)
    assert float(per_view.min()) > 0.5 * float(per_view.max())
    small = torch.full((3, 4, 5), 0.5, dtype=torch.float64)
    assert torch.equal(synth.poisson_log_data(small, 1e4, 9), synth.poisson_log_data(small, 1e4, 9, chunk=60))
