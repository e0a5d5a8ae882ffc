"""mlmc_measure_peaks: the arithmetic throughput probes behind the ALU rooflines.

Sanity bars from the hardware's unit counts (152 SMs, at most ~2.1 GHz): FP32 fused multiply-adds
run on 128 lanes per SM (at most ~40e12 FMA/s, 80 TFLOP/s), special-function operations on a
sixteenth of that, FP64 far slower on this part; INT32 multiply-adds at most at the FP32 rate.
Each measurement must lie below its unit-count ceiling and within a factor of a few of it (or,
for FP64, above a floor), and two calls agree to 10 %.
"""
import pytest
import torch

from paper_1904_00429_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def test_peaks_are_measured_and_plausible():
    a = binding.measure_peaks()
    b = binding.measure_peaks()
    print(f"peaks: {a}")
    ceil_fma = 152 * 128 * 2.2e9
    assert 0.2 * 2 * ceil_fma < a["fp32_flops"] <= 2 * ceil_fma
    assert 1e11 < a["fp64_flops"] < 2 * ceil_fma
    assert 0.05 * ceil_fma < a["int32_imad_per_s"] <= ceil_fma
    assert 0.01 * ceil_fma < a["mufu_sin_per_s"] <= ceil_fma / 4
    for k in a:
        assert abs(a[k] - b[k]) <= 0.1 * max(a[k], b[k]), k
