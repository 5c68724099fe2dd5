"""The on-chip peaks the roofline is held against, measured by the library:
the FP32 FMA rate and the shared-memory load bandwidth must be positive and
lie between a quarter and twice of what the device's unit counts give at a
2.2 GHz clock (128 FP32 lanes x 2 flop and 128 bytes per clock per SM)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2103_10329_gb300 import build
    build.build()


def test_measured_onchip_peaks_are_plausible():
    from paper_2103_10329_gb300 import mgct
    p = mgct.measure_onchip_peaks()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    # the clock under load is at most the boost clock; take 2.2 GHz as a bound
    fp32_max = sms * 128 * 2 * 2.2e9 / 1e12
    lds_max = sms * 128 * 2.2e9 / 1e9
    assert 0.25 * fp32_max < p["fp32_tflops"] <= 2 * fp32_max, p
    assert 0.25 * lds_max < p["lds_gbs"] <= 2 * lds_max, p
