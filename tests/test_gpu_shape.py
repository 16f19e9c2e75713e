"""Crystals of any shape (bpm_set_crystal_shape): the mask Pi(x, y, z) of a
caller replaces the crystal's boundaries (the method is offered for crystals
of arbitrary shape; the geometry follows from the boundaries, end of
Section 2).  GPU against the FP64 oracle, and against the boundary form."""
import numpy as np
import pytest

import oracle.oracle as orc
from paper_2201_08500_gb300 import bpm
from test_gpu_parity import TOL_FIELD, TOL_RINT, deformed_small, errors, run_gpu
from test_gpu_parity import stream  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def odd_shape(w):
    """A tilted front face, a back face that bulges along z, and a round void."""
    nz, nx = w.nz, w.nx
    m = np.zeros((nz, nx), np.uint8)
    x = np.arange(nx) * w.dx
    Z = nz * w.dz
    d = w.thickness
    for n in range(nz):
        z = n * w.dz
        front = w.x_surface + 0.2 * z
        back = w.x_surface + d * (1.0 + 0.3 * np.sin(2 * np.pi * z / Z))
        m[n] = (x >= front) & (x < back)
    zc, xc, rad = 0.5 * Z, w.x_surface + 0.5 * d, 0.15 * d
    zz = (np.arange(nz) * w.dz)[:, None]
    m[(zz - zc) ** 2 + (x[None, :] - xc) ** 2 < rad ** 2] = 0
    return m


def slab_mask(w):
    m = np.zeros((w.nz, w.nx), np.uint8)
    x = np.arange(w.nx) * w.dx
    m[:, (x >= w.x_surface) & (x < w.x_surface + w.thickness)] = 1
    return m


def test_arbitrary_crystal_shape_matches_oracle(stream):
    w = deformed_small(1024, nz=200, n_ch=3, seed=41)
    w.mask = odd_shape(w)
    assert 0 < w.mask.sum() < w.mask.size
    g = run_gpu(w, stream)
    e = errors(w, g)
    assert e["per_ch"] < TOL_FIELD and e["relh"] < TOL_FIELD, e
    rint = g["refl"][2]
    assert abs(rint / orc.integrated_reflectivity(e["oR"], w.omega) - 1) < TOL_RINT
    # the shape matters: the boundary form of the same crystal differs
    w2 = deformed_small(1024, nz=200, n_ch=3, seed=41)
    g2 = run_gpu(w2, stream)
    assert np.linalg.norm(g2["eh"] - g["eh"]) > 1e-3 * np.linalg.norm(g["eh"])


def test_slab_shaped_mask_equals_the_boundaries_bitwise(stream):
    w = deformed_small(2048, nz=80, n_ch=4, seed=42)
    ref = run_gpu(w, stream)
    w.mask = slab_mask(w)
    got = run_gpu(w, stream)
    for k in ("e0", "eh"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.array_equal(got["refl"][0], ref["refl"][0])


def test_shape_given_after_the_crystal_and_cleared_again(stream):
    w = deformed_small(1024, nz=60, n_ch=2, seed=43)
    ref = run_gpu(w, stream)
    mask = odd_shape(w)
    p = bpm.plan_from_workload(w, stream=stream)   # boundaries
    p.set_crystal_shape(mask)                       # rebuilds the deformation factor
    p.set_pulse(w.omega, w.S, w.theta_i, w.x0, w.w0, w.zx, w.zR)
    p.run()
    p.sync()
    shaped = p.eh()
    p.set_crystal_shape(None)                       # back to the boundaries
    p.set_pulse(w.omega, w.S, w.theta_i, w.x0, w.w0, w.zx, w.zR)
    p.run()
    p.sync()
    assert np.array_equal(p.eh(), ref["eh"])
    p.close()
    w.mask = mask
    assert np.array_equal(shaped, run_gpu(w, stream)["eh"])
    with pytest.raises(ValueError):
        q = bpm.plan_from_workload(w, stream=stream)
        try:
            q.set_crystal_shape(np.ones((3, 3), np.uint8))
        finally:
            q.close()


def test_3d_crystal_shape_matches_oracle():
    """3D: a slab whose thickness grows with y (mask [nz][ny][nx])."""
    from test_gpu_3d import case3d
    w = case3d(256, 256, 24, 2, seed=44)
    m = np.zeros((w.nz, w.ny, w.nx), np.uint8)
    x = np.arange(w.nx) * w.dx
    for r in range(w.ny):
        back = w.x_surface + w.thickness * (0.5 + r / w.ny)
        m[:, r, (x >= w.x_surface) & (x < back)] = 1
    w.mask = m
    g = run_gpu(w, None)
    e = errors(w, g)
    assert e["per_ch"] < TOL_FIELD, e
