"""The allocation-free entry point, bpm_run_noalloc, against the plan-based path.

bpm_run_noalloc is for callers that must not allocate device memory while they
run this code (a process whose device memory a caller-side pool owns, or a
latency-bound loop that must not take the allocator's lock).  Its intermediate
buffers live in one fixed device array shared by all calls, so this test makes
two different calls in a row and checks each against bpm_plan_create + bpm_run
on the same inputs.  Both run the same setup and march kernels on the same
inputs, so the results must be bitwise equal (which also holds them within the
parity tolerance of the other GPU tests).  It also checks that a request beyond
the array's limits, and a caller buffer of the wrong size, are refused with a
clear error.  The file is named so that pytest collects it last; it passes
alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_2201_08500_gb300 import bpm, workloads

pytestmark = pytest.mark.gpu

TOL_FIELD = 1e-4
TOL_R = 1e-5


def small_case(nx, nz, n_ch, seed):
    rng = np.random.default_rng(seed)
    dx = 0.5e-6
    xs = (nx * 3 // 8 - 0.5) * dx
    u = workloads.thermal_bump_2d(nx, nz, dx, dx, xs, 0.3 * workloads.D_HKL, nx // 16 * dx)
    u += rng.uniform(-0.02, 0.02, size=u.shape) * workloads.D_HKL
    omega, S = workloads.band(n_ch)
    return workloads.Workload(f"noalloc{nx}", 2, nx, 1, nz, dx, 0.0, dx, workloads.CHI0,
                              workloads.CHIH, workloads.CHIH, workloads.THETA_B,
                              workloads.LAMBDA_B, xs, nx // 8 * dx, u, omega, S,
                              workloads.THETA_B, xs - 40 * dx, 12 * dx)


def plan_path(w, stream):
    p = bpm.plan_from_workload(w, stream=stream)
    p.run()
    p.sync()
    out = p.e0(), p.eh(), p.reflectivity()[0]
    p.close()
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_matches_plan_path_on_two_calls_in_a_row():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    assert 0 < bpm.load().bpm_noalloc_scratch_bytes() < 8 * 1024 * 1024
    cases = [small_case(1024, 300, 8, seed=1), small_case(2048, 200, 5, seed=2)]
    refs = [plan_path(w, stream) for w in cases]
    outs = []
    for w in cases:  # two calls in a row through the shared scratch array
        e0 = torch.empty((w.n_ch, w.nx), dtype=torch.complex64, device="cuda")
        eh = torch.empty_like(e0)
        R = torch.empty(w.n_ch, dtype=torch.float64, device="cuda")
        u = torch.from_numpy(np.ascontiguousarray(w.u)).cuda()
        bpm.run_noalloc(w, e0, eh, R, u_dev=u, stream=stream)
        outs.append((e0, eh, R, u))
    torch.cuda.synchronize()
    for (e0, eh, R, _), (r0, rh, rR) in zip(outs, refs):
        g0, gh, gR = e0.cpu().numpy(), eh.cpu().numpy(), R.cpu().numpy()
        assert rel(g0, r0) < TOL_FIELD and rel(gh, rh) < TOL_FIELD
        assert np.max(np.abs(gR - rR)) < TOL_R
        # same kernels, same inputs: bitwise equal
        assert np.array_equal(g0, r0) and np.array_equal(gh, rh) and np.array_equal(gR, rR)
        assert np.linalg.norm(rh) > 1e-3 * np.linalg.norm(r0)


def test_noalloc_refuses_sizes_beyond_its_array():
    import torch
    torch.cuda.set_device(0)
    w = small_case(1024, 100, 17, seed=3)  # 17 channels > 16
    e0 = torch.empty((w.n_ch, w.nx), dtype=torch.complex64, device="cuda")
    with pytest.raises(bpm.BpmError) as ei:
        bpm.run_noalloc(w, e0, torch.empty_like(e0),
                        torch.empty(w.n_ch, dtype=torch.float64, device="cuda"))
    assert ei.value.status == 4 and "n_channels" in str(ei.value)


def test_noalloc_refuses_a_mis_sized_output_buffer():
    import torch
    torch.cuda.set_device(0)
    w = small_case(1024, 100, 4, seed=4)
    e0 = torch.empty((w.n_ch, w.nx), dtype=torch.complex64, device="cuda")
    short = torch.empty((w.n_ch, w.nx - 1), dtype=torch.complex64, device="cuda")
    R = torch.empty(w.n_ch, dtype=torch.float64, device="cuda")
    with pytest.raises(bpm.BpmError) as ei:
        bpm.run_noalloc(w, e0, short, R)
    assert ei.value.status == 1 and "eh_out" in str(ei.value)
    with pytest.raises(bpm.BpmError):
        bpm.run_noalloc(w, e0, e0, R, u_dev=torch.zeros(w.nz * w.nx - 1, dtype=torch.float64,
                                                          device="cuda"))
