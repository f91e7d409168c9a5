"""The arithmetic-peak probes (bo_measure_alu_peaks) return plausible rates.

They only time register-resident loops; the check is that each rate is
positive and finite and that the units keep their known order on this GPU:
the packed f32x2 FMA at least the scalar one, FP32 far above FP64.
"""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2111_14991_gb300 import build
    build.build()


def test_alu_peaks_plausible():
    import torch
    from paper_2111_14991_gb300 import bo
    torch.cuda.set_device(0)
    r = bo.measure_alu_peaks()
    print("ALU", r)
    for k in ("fp64_fma_tflops", "fp32_fma_tflops", "fp32x2_fma_tflops", "mufu_gops"):
        assert math.isfinite(r[k]) and r[k] > 0, (k, r)
    assert r["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert r["fp32x2_fma_tflops"] >= 0.9 * r["fp32_fma_tflops"]
    assert r["fp32_fma_tflops"] > 4 * r["fp64_fma_tflops"]
