"""Failure detection on the device without a fault: the library's bounded
wait (the one the tensor-core convolutions use for their MMAs) is run on a
barrier nothing ever completes; it must give up after its limit, report it,
and leave the context usable."""
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2103_10329_gb300 import build
    build.build()


def test_bounded_wait_expires_and_reports():
    from paper_2103_10329_gb300 import mgct
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert mgct.check_bounded_wait(0.2)
    dt = time.perf_counter() - t0
    assert 0.15 < dt < 5.0, dt
    # the context is still usable: a convolution pass runs and reports no expiry
    net = mgct.Net(seed=1)
    step = torch.randn((1, 12, 16, 16), device="cuda")
    out = net.apply(step)
    net.check()
    assert torch.isfinite(out).all()
    assert np.isclose(float(torch.sqrt((out.double() ** 2).mean())), float(torch.sqrt((step.double() ** 2).mean())),
                      rtol=1e-5)
