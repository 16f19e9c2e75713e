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


def test_a_bounded_copy_wait_gives_up_and_reports_without_hanging():
    """The kernels that wait on bulk copies (the streamed 3D column pass) bound
    every wait: here one such wait is made to run out on purpose (an mbarrier
    expecting bytes that no copy brings), at a small poll limit.  It must give
    up, record the status, and leave the context usable: a plan runs and
    matches a plan run before the probe."""
    import numpy as np
    import torch
    from paper_2201_08500_gb300 import workloads
    torch.cuda.set_device(0)
    w = workloads.tiny(n_ch=4)
    w.nz = 20
    w.u = None
    before = bpm.plan_from_workload(w)
    before.run()
    before.sync()
    ref = before.eh()
    before.close()
    assert bpm.check_bounded_wait(1 << 10) is True
    after = bpm.plan_from_workload(w)
    after.run()
    after.sync()
    assert np.array_equal(after.eh(), ref)
    after.close()
