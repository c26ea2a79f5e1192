"""The peak probes behind the CUDA-core rooflines (wrf_measure_alu_peaks):
finite, positive, and within the unit-count bounds of a 148-SM part at its
maximum clock (128 FP32 lanes per SM, 2 FLOP per FMA; a two-lane FMA may at
most double that; ex2 is a MUFU operation, far below the FMA rate)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_alu_peaks_are_plausible():
    from paper_2506_12787_b300 import api, build
    build.build()
    assert torch.cuda.is_available()
    fma, fma2, ex2 = api.wrf_measure_alu_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clk = 2.2e9  # above the part's maximum SM clock
    unit = sms * 128 * 2 * clk
    print(f"FP32 fma {fma / 1e12:.1f} TFLOP/s, fma.rn.f32x2 {fma2 / 1e12:.1f} TFLOP/s, "
          f"ex2 {ex2 / 1e12:.2f} T/s")
    assert 0.3 * unit < fma <= unit
    assert 0.3 * unit < fma2 <= 2 * unit
    assert 0 < ex2 < fma / 2
