"""The measured CUDA-core peak (bpm_measure_peak) that the march rooflines
divide by: one launch of FMA chains on every SM must land at or below the
unit-count rate (SMs x 128 FP32 lanes x 2 flop, resp. the FP64 units, per
clock at the maximum clock) and well above a quarter of it for FP32."""
import pytest

from paper_2201_08500_gb300 import bpm

pytestmark = pytest.mark.gpu


def test_fp32_and_fp64_peaks_are_physical():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound32 = sms * 128 * 2 * 2.07e9
    bpm.measure_peak(bpm.BPM_PEAK_FP32, 1 << 10)
    r32, ms32 = bpm.measure_peak(bpm.BPM_PEAK_FP32, 1 << 15)
    assert ms32 > 0 and 0.25 * bound32 < r32 <= 1.02 * bound32, (r32, bound32)
    r64, ms64 = bpm.measure_peak(bpm.BPM_PEAK_FP64, 1 << 8)
    assert ms64 > 0 and 0 < r64 < r32
    with pytest.raises(bpm.BpmError):
        bpm.measure_peak(7, 10)
