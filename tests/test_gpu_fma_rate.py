"""The measured FP32 FMA rate (hmm_fp32_fma_rate), the denominator beside the
derived FP32 peak in the roofline of the FP32 micro kernels.

Bounds: GB300 SMs have 128 FP32 lanes, so scalar FMAs cannot exceed
SMs x 128 x 2 flops x the maximum SM clock; the paired FP32x2 instruction is
given twice that as its ceiling. The floors only catch a broken measurement.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

MAX_SM_MHZ = 2070.0


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_09463_gb300 import build
    build()
    return torch


def test_fp32_fma_rate_within_the_lane_count(torch_cuda):
    from paper_2108_09463_gb300 import fp32_fma_rate
    nsm = torch_cuda.cuda.get_device_properties(0).multi_processor_count
    nominal = nsm * 128 * 2 * MAX_SM_MHZ * 1e6
    scalar = fp32_fma_rate(packed=False)
    packed = fp32_fma_rate(packed=True)
    print(f"FP32 FMA rate: scalar {scalar / 1e12:.1f} TFLOP/s, packed {packed / 1e12:.1f} TFLOP/s, "
          f"lanes x clock {nominal / 1e12:.1f} TFLOP/s")
    assert 0.3 * nominal < scalar < 1.02 * nominal
    assert 0.3 * nominal < packed < 2.04 * nominal


def test_fp32_fma_rate_rejects_bad_arguments(torch_cuda):
    from paper_2108_09463_gb300 import load_library
    lib = load_library()
    out = ctypes.c_double()
    assert lib.hmm_fp32_fma_rate(2, ctypes.byref(out)) == 1
    assert lib.hmm_fp32_fma_rate(1, None) == 1
