"""GPU parity of the 3D (x, y, z) HBM-streamed path against the FP64 oracle."""
import numpy as np
import pytest

import oracle.oracle as orc
from paper_2201_08500_gb300 import bpm, workloads

pytestmark = pytest.mark.gpu

TOL_FIELD = 1e-4


@pytest.fixture(scope="module", autouse=True)
def device():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def case3d(nx, ny, nz, n_ch, seed):
    """3D slab with a 2D Gaussian thermal bump plus roughness; beam just in front."""
    rng = np.random.default_rng(seed)
    dx = dy = 1.0e-6
    dz = 0.25e-6
    xs = (nx * 5 // 16 - 0.5) * dx
    u = workloads.thermal_bump_3d(nx, ny, nz, dx, dy, dz, xs, 0.4 * workloads.D_HKL,
                                  nx // 8 * dx, ny // 6 * dy)
    u += rng.uniform(-0.02, 0.02, size=u.shape) * workloads.D_HKL
    omega, S = workloads.band(max(n_ch, 2))
    omega, S = omega[:n_ch], S[:n_ch]
    return workloads.Workload(f"c3d{nx}x{ny}", 3, nx, ny, nz, dx, dy, dz, workloads.CHI0,
                              workloads.CHIH, workloads.CHIH, workloads.THETA_B,
                              workloads.LAMBDA_B, xs, nx // 8 * dx, u, omega, S,
                              workloads.THETA_B, xs - 8 * dx, 6 * dx)


def gpu(w, steps=None):
    p = bpm.plan_from_workload(w)
    p.run(steps)
    p.sync()
    out = p.e0(), p.eh(), p.reflectivity()[0]
    p.close()
    return out


def check(w, e0, eh, channels=None):
    ws = w if channels is None else w.subset(channels)
    o0, oh, init = orc.run(ws)
    sel = slice(None) if channels is None else np.asarray(channels)
    inc = np.linalg.norm(init, axis=1)
    err = max(np.max(np.linalg.norm(e0[sel] - o0, axis=1) / inc),
              np.max(np.linalg.norm(eh[sel] - oh, axis=1) / inc))
    assert err < TOL_FIELD, err
    assert np.linalg.norm(oh) > 1e-3 * np.linalg.norm(init)
    return o0, oh, init


@pytest.mark.parametrize("nx,ny,nz", [(256, 256, 40), (512, 256, 24), (256, 1024, 12)])
def test_3d_matches_oracle(nx, ny, nz):
    w = case3d(nx, ny, nz, 2, seed=nx + ny)
    e0, eh, R = gpu(w)
    o0, oh, init = check(w, e0, eh)
    oR, _ = orc.reflectivity(init, o0, oh)
    assert np.max(np.abs(R - oR)) < 1e-5


def test_3d_split_run_is_bitwise_identical():
    w = case3d(256, 256, 30, 2, seed=4)
    e0, eh, _ = gpu(w)
    p = bpm.plan_from_workload(w)
    p.run(11)
    p.run(19)
    p.sync()
    assert np.array_equal(p.e0(), e0) and np.array_equal(p.eh(), eh)
    p.close()


def test_3d_y_uniform_field_equals_2d_path():
    """A y-independent field in a y-independent crystal evolves as the 2D problem."""
    ny, nx, nz = 256, 512, 40
    w3 = case3d(nx, ny, nz, 1, seed=2)
    w3.u = None
    dx = w3.dx
    w2 = workloads.Workload("y-flat", 2, nx, 1, nz, dx, 0.0, w3.dz, w3.chi0, w3.chih, w3.chihb,
                            w3.theta_B, w3.lambda_B, w3.x_surface, w3.thickness, None, w3.omega,
                            w3.S, w3.theta_i, w3.x0, w3.w0)
    p2 = bpm.plan_from_workload(w2)
    inc2 = p2.e0()
    p2.run()
    e2, h2 = p2.e0(), p2.eh()
    p2.close()
    p3 = bpm.plan_from_workload(w3)
    f0 = np.tile(inc2[0], ny)[None, :].astype(np.complex64)
    p3.set_fields(f0, np.zeros_like(f0), 0)
    p3.run()
    e3 = p3.e0().reshape(ny, nx)
    h3 = p3.eh().reshape(ny, nx)
    p3.close()
    scale = np.linalg.norm(inc2)
    assert np.max(np.linalg.norm(e3 - e2[0], axis=1)) / scale < 1e-5
    assert np.max(np.linalg.norm(h3 - h2[0], axis=1)) / scale < 1e-5


def test_3d_full_transverse_grid_sampled_channel():
    """The bench's 3D launch configuration (512 x 512, all 128 channels), 40 of
    the 1000 steps, one channel at the band centre against the oracle."""
    w = workloads.large_3d(nz=40)
    w.x0 = w.x_surface - 6 * w.dx  # the beam reaches the crystal within the 40 steps
    e0, eh, _ = gpu(w)
    check(w, e0, eh, channels=[64])
    assert np.all(np.isfinite(e0)) and np.all(np.isfinite(eh))


def test_3d_rejects_unsupported_sizes():
    with pytest.raises(bpm.BpmError):
        bpm.Plan(3, 2048, 256, 10, 1e-6, 1e-6, 1e-6, 1)


def test_3d_asymmetric_cut_matches_oracle():
    import math
    w = case3d(256, 256, 30, 1, seed=11)
    w.tan_psi = math.tan(math.radians(7.0))
    e0, eh, _ = gpu(w)
    check(w, e0, eh)


def test_3d_zero_steps_return_the_incident_field():
    """The empty 3D march: run(0) leaves E0 at the incident beam and Eh at zero."""
    w = case3d(256, 256, 8, 2, seed=9)
    p = bpm.plan_from_workload(w)
    p.run(0)
    p.sync()
    e0, eh = p.e0(), p.eh()
    R, T, rint = p.reflectivity()
    _, _, init = orc.run(w, n_steps=0)
    inc = np.linalg.norm(init, axis=1)
    assert np.max(np.linalg.norm(e0.reshape(init.shape) - init, axis=1) / inc) < 1e-6
    assert not np.any(eh) and not np.any(R) and rint == 0.0
    assert np.max(np.abs(T - 1.0)) < 1e-6
    p.close()
