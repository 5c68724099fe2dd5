"""Learned correction network on the GPU (BF16 tensor-core convolutions,
float32 accumulation) against the FP64 oracle of the same network.

Tolerance, from the arithmetic: the GPU stores the input, the weights, the
hidden activations and the back-propagated gradients in bfloat16 (unit
roundoff u = 2^-9) and accumulates in float32.  The oracle with bf16=True
rounds the same tensors at the same places, so what remains is the float32
accumulation order and the occasional different rounding of a value that
falls near a bf16 rounding boundary: errors of a few u relative to the
largest entry.  The bound used is 8u = 1.6 %."""
import numpy as np
import pytest
import torch

from oracle import learned as NL
from tests.helpers import to_np

pytestmark = pytest.mark.gpu
U = 2.0 ** -9


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2103_10329_gb300 import build
    build.build()


def random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    layers = []
    for ci, co in zip(NL.CIN, NL.COUT):
        sd = scale * np.sqrt(2.0 / (27 * ci))
        layers.append((rng.standard_normal((27, co, ci)) * sd, rng.standard_normal(co) * 0.1))
    return NL.pack(layers).astype(np.float32)


def test_param_layout_roundtrip():
    from paper_2103_10329_gb300 import mgct
    net = mgct.Net(seed=3)
    assert net.count == NL.param_count()
    p = random_params(1)
    net.set_params(p)
    np.testing.assert_array_equal(net.params(), p)
    # the default initialisation has a zero output layer: no correction
    net0 = mgct.Net(seed=4)
    step = torch.randn((1, 8, 9, 10), device="cuda")
    out = net0.apply(step)
    torch.cuda.synchronize()
    assert torch.allclose(out, step, rtol=1e-6, atol=0)


@pytest.mark.parametrize("shape", [(1, 16, 16, 16), (2, 7, 12, 19)])
def test_forward_vs_oracle(shape):
    from paper_2103_10329_gb300 import mgct
    net = mgct.Net()
    p = random_params(5)
    net.set_params(p)
    step = 0.01 * np.random.default_rng(6).standard_normal(shape)
    out = to_np(net.apply(torch.tensor(step, dtype=torch.float32, device="cuda")))
    net.check()
    s = np.sqrt(np.mean(step.astype(np.float32).astype(np.float64) ** 2))
    x = step.astype(np.float32).astype(np.float64) / s
    y_bf, _ = NL.forward(p.astype(np.float64), x, bf=True)
    y_64, _ = NL.forward(p.astype(np.float64), x, bf=False)
    y_gpu = out / s - x
    scale = np.abs(y_64).max()
    assert np.abs(y_gpu - y_bf).max() <= 8 * U * scale
    assert np.abs(y_gpu - y_64).max() <= 32 * U * scale


@pytest.mark.parametrize("slab", [1, 5, 13])
def test_slabwise_apply_equals_whole_volume(slab):
    """z-slabs with a 4-plane halo give the whole-volume result bit for bit
    (each voxel's sums run in the same order; the RMS is the whole volume's)."""
    from paper_2103_10329_gb300 import mgct
    net = mgct.Net()
    net.set_params(random_params(31))
    g = torch.Generator(device="cuda").manual_seed(32)
    step = 0.01 * torch.randn((2, 40, 33, 29), device="cuda", generator=g)
    full = net.apply(step).clone()
    part = net.apply(step, slab_planes=slab)
    net.check()
    assert torch.equal(full, part)


@pytest.mark.parametrize("shape", [(2, 20, 70, 45), (1, 256, 256, 256), (1, 1024, 1024, 1024)],
                         ids=["ragged", "256", "1024"])
def test_forward_sampled_large(shape):
    """Volumes of many brick tiles (ragged in every axis; the 256^3 grid the
    correction runs on in the bench, and the 1024^3 evaluation volume, which
    runs in z-slabs), checked at sampled voxels: the four 3x3x3 layers see
    the input within 4 voxels, so the oracle on the 9^3 crop around a voxel
    (cut at the volume's own faces, where the zero padding is the same)
    gives that voxel's output exactly."""
    from paper_2103_10329_gb300 import mgct
    net = mgct.Net()
    p = random_params(21)
    net.set_params(p)
    g = torch.Generator(device="cuda").manual_seed(22)
    step = 0.01 * torch.randn(shape, device="cuda", generator=g)
    out = net.apply(step)
    net.check()
    s = float(torch.sqrt((step.double() ** 2).sum() / step.numel()))
    rng = np.random.default_rng(23)
    B, D, H, W = shape
    pts = [tuple(int(rng.integers(0, n)) for n in (B, D, H, W)) for _ in range(48)]
    pts += [(0, 0, 0, 0), (B - 1, D - 1, H - 1, W - 1), (0, D - 1, 0, W - 1)]
    pw = p.astype(np.float64)
    errs, mags = [], []
    for b, z, y, x in pts:
        lo = [max(0, c - 4) for c in (z, y, x)]
        hi = [min(n, c + 5) for c, n in zip((z, y, x), (D, H, W))]
        crop = to_np(step[b, lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]).astype(np.float64) / s
        yb, _ = NL.forward(pw, crop[None], bf=True)
        ref = yb[0, z - lo[0], y - lo[1], x - lo[2]]
        got = float(out[b, z, y, x]) / s - crop[z - lo[0], y - lo[1], x - lo[2]]
        errs.append(abs(got - ref))
        mags.append(abs(ref))
    assert max(errs) <= 8 * U * max(max(mags), 1.0), (max(errs), max(mags))


def _grad_magnitudes(params, x, t):
    """Per-entry magnitude of each gradient sum, |g| * |a| summed over the
    voxels: the scale of its rounding error.  It runs the oracle's own
    forward pass and convolution routines (bf16 storage emulated) on absolute
    values; the expected gradients themselves come from loss_and_grads."""
    r = NL.bf16
    y, (layers, acts) = NL.forward(params, x, bf=True)
    res = x + y - t
    g = r((2.0 / res.size) * res)[..., None]
    mags = [None] * 4
    for l in range(3, -1, -1):
        w, _ = layers[l]
        mags[l] = (NL.conv_weight_grad(np.abs(acts[l]), np.abs(g)), np.abs(g).sum(axis=(0, 1, 2, 3)))
        if l > 0:
            g = r(NL.conv_data_grad(g, w) * (acts[l] > 0))
    return mags


def test_gradients_vs_oracle():
    """Weight and bias gradients entry by entry.  Each entry is a sum over
    voxels of a back-propagated gradient times an activation, both stored in
    bf16 on the GPU and rounded at the same places by the oracle; they differ
    only where float32 accumulation order moves a value across a bf16
    rounding boundary (one bf16 step, 2u, at rare voxels) and by the float32
    summation error (~1e-6 relative).  A ReLU whose float32 pre-activation
    lies within the accumulation error of zero may also switch, which moves
    the activation by that error alone (~1e-6 of the layer's scale): an
    absolute floor of 1e-5 of the layer's largest magnitude covers it, where
    a channel is almost never active.  So every entry must lie within
    4u * sum_p |g_p| |a_p| + 1e-5 * max of the oracle: a wrong tap, channel
    or layer moves an entry by a few percent of its magnitude at random
    data."""
    from paper_2103_10329_gb300 import mgct
    net = mgct.Net()
    p = random_params(7)
    net.set_params(p)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((2, 10, 12, 14))
    t = x + 0.5 * rng.standard_normal(x.shape)
    xf, tf = x.astype(np.float32), t.astype(np.float32)
    loss = net.forward_backward(torch.tensor(xf, device="cuda"), torch.tensor(tf, device="cuda"))
    g_gpu = net.grads().astype(np.float64)
    pw, xw, tw = p.astype(np.float64), xf.astype(np.float64), tf.astype(np.float64)
    l_ref, g_ref = NL.loss_and_grads(pw, xw, tw, bf=True)
    assert abs(loss.item() - l_ref) <= 8 * U * l_ref
    mags = _grad_magnitudes(pw, xw, tw)
    layers_gpu = NL.unpack(g_gpu)
    layers_ref = NL.unpack(g_ref)
    for l, ((wg, bg), (wr, br), (wm, bm)) in enumerate(zip(layers_gpu, layers_ref, mags)):
        wtol = 4 * U * wm + 1e-5 * wm.max()
        btol = 4 * U * bm + 1e-5 * bm.max()
        ew = np.abs(wg - wr) / wtol
        eb = np.abs(bg - br) / btol
        assert ew.max() <= 1.0, (l, "weights", float(ew.max()), np.unravel_index(ew.argmax(), ew.shape))
        assert eb.max() <= 1.0, (l, "bias", float(eb.max()))
        # and the layer as a whole, relative to its own norm
        assert np.linalg.norm(wg - wr) <= 8 * U * np.linalg.norm(wr), l
        # the bound is sharp enough to see a wrong tap: with two taps of the
        # oracle's gradient swapped, most entries of those taps break it
        swapped = wr[[1, 0] + list(range(2, 27))]
        assert (np.abs(wg - swapped)[:2] > wtol[:2]).mean() > 0.5, l


def test_adam_step():
    from paper_2103_10329_gb300 import mgct
    net = mgct.Net()
    p = random_params(9)
    net.set_params(p)
    rng = np.random.default_rng(10)
    x = torch.tensor(rng.standard_normal((1, 8, 8, 8)), dtype=torch.float32, device="cuda")
    t = x + 0.3
    net.forward_backward(x, t)
    g = net.grads().astype(np.float64)
    net.adam_step(1e-3)
    q = net.params().astype(np.float64)
    # first Adam step: m = 0.1 g, v = 0.001 g^2, bias corrections 0.1 and 0.001
    want = p.astype(np.float64) - 1e-3 * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(q, want, rtol=1e-5, atol=1e-7)


def test_deterministic_training_step():
    from paper_2103_10329_gb300 import mgct
    rng = np.random.default_rng(11)
    x = torch.tensor(rng.standard_normal((2, 9, 9, 9)), dtype=torch.float32, device="cuda")
    t = 0.5 * x
    outs = []
    for _ in range(2):
        net = mgct.Net(seed=12)
        net.set_params(random_params(13))
        for _ in range(3):
            net.forward_backward(x, t)
            net.adam_step(1e-3)
        net.check()
        outs.append(net.params())
    np.testing.assert_array_equal(outs[0], outs[1])
