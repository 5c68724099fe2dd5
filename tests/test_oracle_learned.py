"""Pins for the FP64 oracle of the learned correction network (CPU)."""
import numpy as np
import scipy.ndimage
import torch

from oracle import learned as NL


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(NL.param_count()) * 0.1
    x = rng.standard_normal((2, 4, 5, 6))
    t = rng.standard_normal((2, 4, 5, 6))
    _, g = NL.loss_and_grads(p, x, t)
    for i in rng.choice(len(p), 25, replace=False):
        e = 1e-6
        p1, p2 = p.copy(), p.copy()
        p1[i] += e
        p2[i] -= e
        fd = (NL.loss_and_grads(p1, x, t)[0] - NL.loss_and_grads(p2, x, t)[0]) / (2 * e)
        assert abs(g[i] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, g[i], fd)


def test_conv_equals_library_correlation():
    """One output channel of conv() from one input channel equals scipy's
    constant-mode correlation with that tap kernel."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 6, 7, 8, 3))
    w = rng.standard_normal((27, 2, 3))
    out = NL.conv(x, w)
    for co in range(2):
        ref = np.zeros((6, 7, 8))
        for ci in range(3):
            k = w[:, co, ci].reshape(3, 3, 3)  # [dz][dy][dx] = tap order
            ref += scipy.ndimage.correlate(x[0, ..., ci], k, mode="constant", cval=0.0)
        np.testing.assert_allclose(out[0, ..., co], ref, atol=1e-12)


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(2).standard_normal(10000) * 10.0 ** np.random.default_rng(3).integers(-8, 8, 10000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(NL.bf16(x), ref)


def test_zero_output_layer_predicts_no_correction():
    rng = np.random.default_rng(4)
    layers = NL.unpack(rng.standard_normal(NL.param_count()))
    layers[3] = (np.zeros_like(layers[3][0]), np.zeros_like(layers[3][1]))
    y, _ = NL.forward(NL.pack(layers), rng.standard_normal((1, 4, 4, 4)))
    assert np.abs(y).max() == 0.0
