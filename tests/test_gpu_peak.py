"""The FP32 peak the benchmark divides by: the library's FMA-chain kernel
(fea_fp32_peak) must report a figure between half and 1.1 times the FP32
units' rate at the maximum SM clock (SMs x 128 lanes x 2 x clock)."""
import pytest
import torch

from paper_2005_05899_b300 import fea

pytestmark = pytest.mark.gpu


def test_fp32_peak_against_unit_count():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    ctx = fea.Context(0)
    try:
        ffma, ffma2 = ctx.fp32_peak()
    finally:
        ctx.close()
    props = torch.cuda.get_device_properties(0)
    # the clock is not exposed by torch; 2.1 GHz bounds B300's maximum SM clock
    ceiling = props.multi_processor_count * 128 * 2 * 2.1e9 / 1e12
    for v in (ffma, ffma2):
        assert 0.5 * ceiling * 0.9 < v < 1.1 * ceiling, (v, ceiling)
