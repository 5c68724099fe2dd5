"""The least-squares preconditioner fit (host logic), on the CPU."""
import numpy as np
import scipy.ndimage

import oracle as O
from paper_2103_10329_gb300 import psf


def residual(k, h):
    d = np.zeros_like(h)
    c = h.shape[0] // 2
    d[c, c, c] = 1.0
    r = scipy.ndimage.correlate(h, k, mode="constant")
    # the best scale of k for this h (the line search sets the scale in use)
    a = float(np.sum(r * d) / np.sum(r * r))
    return float(np.linalg.norm(a * r - d))


def synthetic_psf(m=9, s=0.9, az=0.6):
    """A blur of the shape A^T A has: slowly decaying, wider in x/y than in z."""
    g = np.indices((m, m, m)).astype(float) - m // 2
    r = np.sqrt((g[1] ** 2 + g[2] ** 2) / s ** 2 + g[0] ** 2 / az ** 2)
    return 1.0 / (1.0 + r)


def test_delta_psf_gives_delta_kernel():
    h = np.zeros((7, 7, 7))
    h[3, 3, 3] = 1.0
    k = psf.fit_kernel(h)
    d = np.zeros((3, 3, 3))
    d[1, 1, 1] = 1.0
    np.testing.assert_allclose(k, d, atol=1e-12)


def test_fit_is_symmetric_and_beats_eq5():
    """The fitted kernel has the trajectory's symmetries, and -- Eq. 5 lying in
    the same six-class space -- deconvolves the PSF at least as well as Eq. 5
    at its best scale (least squares over that space)."""
    h = synthetic_psf()
    k = psf.fit_kernel(h)
    np.testing.assert_allclose(k, k[::-1, :, :], atol=1e-12)
    np.testing.assert_allclose(k, k[:, ::-1, :], atol=1e-12)
    np.testing.assert_allclose(k, k[:, :, ::-1], atol=1e-12)
    np.testing.assert_allclose(k, np.transpose(k, (0, 2, 1)), atol=1e-12)
    assert residual(k, h) <= residual(O.eq5_kernel(2), h) + 1e-12
    assert residual(k, h) < 0.9 * residual(np.pad(np.ones((1, 1, 1)), 1), h)
