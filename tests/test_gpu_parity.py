"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP32 fields vs the FP64 oracle):
  * per channel, ||A_gpu - A_oracle|| / ||A+(z=0)|| <= 1e-4 for both envelopes
    (the scheme is linear in the incident field, so its norm is the natural
    scale; a relative error of a nearly extinguished field is ill-conditioned);
  * per field over all channels, ||A_gpu - A_oracle||_F / ||A_oracle||_F <= 1e-4;
  * integrated reflectivity R_int: relative error <= 1e-5;
  * time response: relative L2 <= 1e-4.
Runs that repeat the same GPU computation (split runs, channel subsets) must be
bitwise identical.
"""
import numpy as np
import pytest

import oracle.oracle as orc
from paper_2201_08500_gb300 import bpm, workloads

pytestmark = pytest.mark.gpu

TOL_FIELD = 1e-4
TOL_RINT = 1e-5


@pytest.fixture(scope="module")
def stream():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    return torch.cuda.current_stream()


def run_gpu(w, stream, steps=None):
    p = bpm.plan_from_workload(w, stream=stream)
    p.run(steps)
    p.sync()
    out = dict(e0=p.e0(), eh=p.eh(), refl=p.reflectivity())
    if steps is None or steps == w.nz:
        out["time"] = p.eh_time()
    p.close()
    return out


def errors(w, g, channels=None):
    ws = w if channels is None else w.subset(channels)
    o0, oh, init = orc.run(ws)
    sel = slice(None) if channels is None else np.asarray(channels)
    e0, eh = g["e0"][sel], g["eh"][sel]
    inc = np.linalg.norm(init, axis=1)
    per_ch = max(np.max(np.linalg.norm(e0 - o0, axis=1) / inc),
                 np.max(np.linalg.norm(eh - oh, axis=1) / inc))
    rel0 = np.linalg.norm(e0 - o0) / np.linalg.norm(o0)
    relh = np.linalg.norm(eh - oh) / np.linalg.norm(oh)
    oR, oT = orc.reflectivity(init, o0, oh)
    return dict(per_ch=per_ch, rel0=rel0, relh=relh, oR=oR, oT=oT, oh=oh, init=init)


def deformed_small(nx, nz, n_ch, seed=0):
    """A deformed crystal of width nx (thermal bump plus seeded roughness)."""
    rng = np.random.default_rng(seed)
    dx = 0.5e-6
    xs = (nx * 3 // 8 - 0.5) * dx
    d = nx // 8 * dx
    u = workloads.thermal_bump_2d(nx, nz, dx, dx, xs, 0.4 * workloads.D_HKL, nx // 16 * dx)
    u += rng.uniform(-0.02, 0.02, size=u.shape) * workloads.D_HKL
    omega, S = workloads.band(n_ch)
    # beam 40 cells in front of the entrance surface: it reaches the crystal
    # after ~40 steps at 45 degrees, so both envelopes carry power at the end
    return workloads.Workload(f"small{nx}", 2, nx, 1, nz, dx, 0.0, dx, workloads.CHI0,
                              workloads.CHIH, workloads.CHIH, workloads.THETA_B,
                              workloads.LAMBDA_B, xs, d, u, omega, S, workloads.THETA_B,
                              xs - 40 * dx, 12 * dx)


def test_tiny_configuration_all_channels(stream):
    """Nx = 256, 200 steps, 64 channels: every channel and the time response."""
    w = workloads.tiny()
    g = run_gpu(w, stream)
    e = errors(w, g)
    assert e["per_ch"] < TOL_FIELD and e["rel0"] < TOL_FIELD and e["relh"] < TOL_FIELD, e
    R, T, rint = g["refl"]
    o_rint = orc.integrated_reflectivity(e["oR"], w.omega)
    assert abs(rint / o_rint - 1) < TOL_RINT
    assert np.max(np.abs(R - e["oR"])) < 1e-5 and np.max(np.abs(T - e["oT"])) < 1e-5
    ot = orc.omega_to_t(e["oh"], orc.channel_spacing(w.omega))
    assert np.linalg.norm(g["time"] - ot) / np.linalg.norm(ot) < TOL_FIELD


@pytest.mark.parametrize("nx", [256, 512, 1024, 2048, 4096, 8192])
def test_every_transform_size_deformed(stream, nx):
    w = deformed_small(nx, nz=160, n_ch=5, seed=nx)
    g = run_gpu(w, stream)
    e = errors(w, g)
    assert e["per_ch"] < TOL_FIELD and e["rel0"] < TOL_FIELD and e["relh"] < TOL_FIELD, e


@pytest.mark.parametrize("nx,extra", [(256, 7), (512, 3), (1024, 1), (2048, 1)])
def test_grouped_launch_with_ragged_tail(stream, nx, extra):
    """Enough channels that several channels share a block, plus a ragged tail."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    group = {256: 16, 512: 8, 1024: 4, 2048: 2}[nx]
    n_ch = group * sms + extra
    w = deformed_small(nx, nz=24, n_ch=n_ch, seed=3)
    p = bpm.plan_from_workload(w, stream=stream)
    assert p.stats()["channels_per_block"] == group
    p.run()
    p.sync()
    g = dict(e0=p.e0(), eh=p.eh())
    p.close()
    pick = [0, 1, group - 1, group, n_ch // 2, n_ch - 2, n_ch - 1]
    e = errors(w, g, channels=pick)
    assert e["per_ch"] < TOL_FIELD, e


def test_split_run_and_resume_are_bitwise_identical(stream):
    w = deformed_small(1024, nz=120, n_ch=6, seed=9)
    straight = run_gpu(w, stream)
    p = bpm.plan_from_workload(w, stream=stream)
    p.run(47)
    mid0, midh = p.e0(), p.eh()
    p.run(73)
    p.sync()
    assert np.array_equal(p.e0(), straight["e0"]) and np.array_equal(p.eh(), straight["eh"])
    p.close()
    q = bpm.plan_from_workload(w, stream=stream)
    q.set_fields(mid0, midh, 47)
    q.run(73)
    q.sync()
    assert np.array_equal(q.e0(), straight["e0"]) and np.array_equal(q.eh(), straight["eh"])
    assert np.array_equal(q.reflectivity()[0], straight["refl"][0])
    q.close()


def test_channel_alone_equals_channel_in_batch(stream):
    w = deformed_small(512, nz=80, n_ch=12, seed=4)
    full = run_gpu(w, stream)
    for c in (0, 7, 11):
        one = run_gpu(w.subset([c]), stream)
        assert np.array_equal(one["e0"][0], full["e0"][c])
        assert np.array_equal(one["eh"][0], full["eh"][c])


def test_device_tensors_in_and_out(stream):
    import torch
    w = deformed_small(2048, nz=60, n_ch=3, seed=5)
    host = run_gpu(w, stream)
    u_dev = torch.from_numpy(np.ascontiguousarray(w.u)).cuda()
    p = bpm.plan_from_workload(w, stream=stream, u=u_dev)
    p.run()
    e0 = torch.empty((w.n_ch, w.nx), dtype=torch.complex64, device="cuda")
    p.fetch(bpm.BPM_FIELD_E0, out=e0)
    assert np.array_equal(e0.cpu().numpy(), host["e0"])
    p.close()


def test_invalid_arguments_raise(stream):
    w = workloads.tiny(n_ch=2)
    with pytest.raises(bpm.BpmError):
        bpm.Plan(2, 300, 1, 10, 1e-6, 0, 1e-6, 2, stream=stream)  # not a power of two
    p = bpm.plan_from_workload(w, stream=stream)
    with pytest.raises(bpm.BpmError):
        p.run(w.nz + 1)
    p.run(10)
    with pytest.raises(bpm.BpmError):
        p.eh_time()  # march not at nz yet
    with pytest.raises(bpm.BpmError):
        p.fetch(bpm.BPM_FIELD_E0, out=np.empty((1, w.nx), np.complex64))
    p.close()
    q = bpm.Plan(2, 256, 1, 10, 0.5e-6, 0, 0.5e-6, 1, stream=stream)
    with pytest.raises(bpm.BpmError):
        q.run(1)  # no crystal / pulse yet
    with pytest.raises(bpm.BpmError):
        q.set_crystal(0j, 0j, 0j, np.radians(86.0), 1e-10, 0.0, 1e-6)
    q.close()


def test_deformed_full_size_sampled_channels(stream):
    """The bench workload (Nx = 4096, 2000 steps, 1024 channels, thermal bump) in
    the launch configuration the bench times; 4 channels across the band are
    compared with the oracle over the full march."""
    w = workloads.deformed()
    g = run_gpu(w, stream)
    pick = [0, 340, 512, 1023]
    e = errors(w, g, channels=pick)
    assert e["per_ch"] < TOL_FIELD, e
    # each field over the sampled channels, relative to its own norm
    assert e["rel0"] < TOL_FIELD and e["relh"] < TOL_FIELD, e
    R = g["refl"][0]
    assert np.max(np.abs(R[pick] - e["oR"])) < 1e-5
    assert np.all(np.isfinite(g["e0"])) and np.all(np.isfinite(g["eh"]))


@pytest.mark.parametrize("nx", [512, 4096])
def test_strang_splitting_matches_oracle(stream, nx):
    """Second-order splitting (Eq. split-op with a = (0, 1), b = (1/2, 1/2))."""
    w = deformed_small(nx, nz=140, n_ch=3, seed=nx + 1)
    w.split_order = 2
    g = run_gpu(w, stream)
    e = errors(w, g)
    assert e["per_ch"] < TOL_FIELD and e["relh"] < TOL_FIELD, e
    w1 = deformed_small(nx, nz=140, n_ch=3, seed=nx + 1)
    g1 = run_gpu(w1, stream)
    assert np.linalg.norm(g1["eh"] - g["eh"]) > 1e-4 * np.linalg.norm(g["eh"])  # a different scheme


@pytest.mark.parametrize("psi_deg", [6.0, -10.0])
def test_asymmetric_bragg_geometry_matches_oracle(stream, psi_deg):
    import math
    w = deformed_small(2048, nz=200, n_ch=3, seed=7)
    w.tan_psi = math.tan(math.radians(psi_deg))
    g = run_gpu(w, stream)
    e = errors(w, g)
    assert e["per_ch"] < TOL_FIELD and e["relh"] < TOL_FIELD, e


def test_laue_slab_geometry_matches_oracle(stream):
    w = deformed_small(1024, nz=220, n_ch=4, seed=8)
    w.x_surface, w.thickness = -1.0, 2.0  # crystal across the whole x range ...
    w.z_begin, w.z_end = 40.5 * w.dz, 170.5 * w.dz  # ... between two z planes
    g = run_gpu(w, stream)
    e = errors(w, g)
    assert e["per_ch"] < TOL_FIELD and e["relh"] < TOL_FIELD, e


@pytest.mark.parametrize("nx", [512, 4096, 8192])
def test_fourth_order_splitting_matches_oracle(stream, nx):
    """Fourth-order splitting (Eq. split-op, t = 1/(2 - 2^(1/3))): three
    propagations and four couplings per step, two table sets per channel."""
    w = deformed_small(nx, nz=100, n_ch=3, seed=nx + 2)
    w.split_order = 4
    g = run_gpu(w, stream)
    e = errors(w, g)
    assert e["per_ch"] < TOL_FIELD and e["relh"] < TOL_FIELD, e
    w2 = deformed_small(nx, nz=100, n_ch=3, seed=nx + 2)
    w2.split_order = 2
    g2 = run_gpu(w2, stream)
    assert np.linalg.norm(g2["eh"] - g["eh"]) > 1e-5 * np.linalg.norm(g["eh"])  # a different scheme


def test_fourth_order_grouped_channels(stream):
    """Several channels per block at N = 512 with a ragged tail (fourth-order
    plans in batches: test_gpu_batch.py)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    w = deformed_small(512, nz=30, n_ch=8 * sms + 5, seed=12)
    w.split_order = 4
    p = bpm.plan_from_workload(w, stream=stream)
    assert p.stats()["channels_per_block"] == 8
    p.run()
    p.sync()
    g = dict(e0=p.e0(), eh=p.eh())
    e = errors(w, g, channels=[0, 7, 8, w.n_ch - 1])
    assert e["per_ch"] < TOL_FIELD, e
    p.close()


def test_strain_gradient_benchmark(stream):
    """Section 3.2, constant strain gradient: the CUDA path against the oracle
    on the Si(444) case (Nx = 4096, 1800 steps), and the fraction of the new
    branch against exp(-2 pi beta_c/|beta|) = 0.2651 at 1.5e-3 relative."""
    w = workloads.strain_gradient()
    g = run_gpu(w, stream)
    e = errors(w, g)
    assert e["per_ch"] < TOL_FIELD, e
    x = np.arange(w.nx) * w.dx
    inten = np.abs(g["e0"][0]) ** 2 + np.abs(g["eh"][0]) ** 2
    p0 = np.sum(np.abs(e["init"][0]) ** 2)
    trans = np.sum(inten[x >= w.meta["x_back"]]) / p0
    assert abs(trans / w.meta["interbranch"] - 1.0) < 1.5e-3, trans


@pytest.mark.parametrize("form", [0, 3])
def test_zero_steps_return_the_incident_field(stream, form):
    """The empty march: run(0) leaves E0 at the incident beam (Section 3.1) and
    Eh at zero, so R = 0 and T = 1; the remaining steps then give the full
    march.  A plan of no channels is refused."""
    w = deformed_small(2048, nz=30, n_ch=3, seed=5)
    p = bpm.plan_from_workload(w, stream=stream)
    p.set_launch(form=form, channels_per_block=1)
    p.run(0)
    p.sync()
    e0, eh = p.e0(), p.eh()
    R, T, rint = p.reflectivity()
    _, _, init = orc.run(w, n_steps=0)
    inc = np.linalg.norm(init, axis=1)
    assert np.max(np.linalg.norm(e0 - init, axis=1) / inc) < 1e-6
    assert not np.any(eh) and not np.any(R) and rint == 0.0
    assert np.max(np.abs(T - 1.0)) < 1e-6
    p.run(w.nz)
    p.sync()
    e = errors(w, dict(e0=p.e0(), eh=p.eh()))
    assert e["per_ch"] < TOL_FIELD, e
    p.close()
    with pytest.raises(bpm.BpmError):
        bpm.Plan(2, 256, 1, 10, 0.5e-6, 0, 0.5e-6, 0, stream=stream)
