"""The measured FMA rate reported beside the roofline: positive, below the
unit-count figure (SMs x 128 lanes x 2 flops at the maximum SM clock) and
well above half of it on an idle GPU; NULL output is an argument error."""
import ctypes

import pytest

from paper_2106_12655_gb300 import lk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_12655_gb300 import build as B

    B.build()
    lk.load()


def test_measured_fma_rate_is_below_the_unit_count_figure():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = sms * 128 * 2 * 2070e6 / 1e12
    tflops, ms = lk.lk_measure_fp32_peak()
    assert 0.5 * derived < tflops <= 1.02 * derived
    assert ms > 0.0
    st = lk.load().lk_measure_fp32_peak(None, None, None)
    assert st == lk.LK_ERR_ARG
    assert ctypes.c_int(st).value != lk.LK_OK
