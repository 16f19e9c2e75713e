"""Launch forms and their autotuner (bpm_tune): every form computes bitwise the
same fields (only the layout of the work on the GPU differs), the tuner keeps
the fastest measured form, and later plans of the shape use it."""
import numpy as np
import pytest

import oracle.oracle as orc
from paper_2201_08500_gb300 import bpm, workloads
from test_gpu_parity import deformed_small, errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def device():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    bpm.tune_clear()
    yield
    bpm.tune_clear()


def fields(w, **form):
    p = bpm.plan_from_workload(w)
    if form:
        p.set_launch(**form)
    got = p.launch()
    p.run()
    p.sync()
    out = dict(e0=p.e0(), eh=p.eh(), R=p.reflectivity()[0])
    p.close()
    return out, got


@pytest.mark.parametrize("nx,n_ch", [(1024, 611), (2048, 310), (4096, 160), (8192, 40)])
def test_every_2d_form_gives_identical_fields(nx, n_ch):
    """Shared-memory (G = 1 and the maximum), L2, parked and parked-TMEM forms
    (at 1024 two channels per block: 611 channels leave the last block one)."""
    w = deformed_small(nx, nz=48, n_ch=n_ch, seed=31)
    maxg = {1024: 4, 2048: 2, 4096: 1, 8192: 1}[nx]
    ref, _ = fields(w, form=0, channels_per_block=1)
    forms = [dict(form=0, channels_per_block=maxg)]
    if nx <= 4096:
        forms.append(dict(form=1, channels_per_block=maxg))
        forms.append(dict(form=2, channels_per_block=1))
    if nx >= 2048:
        forms.append(dict(form=3, channels_per_block=1))
    if nx == 1024:  # tensor-memory tables, two channels per block
        forms.append(dict(form=3, channels_per_block=2))
    for f in forms:
        got, used = fields(w, **f)
        assert used["form"] == f["form"] and used["channels_per_block"] == f["channels_per_block"]
        for k in ("e0", "eh", "R"):
            assert np.array_equal(got[k], ref[k]), (f, k)
    e = errors(w, ref, channels=[0, n_ch // 2, n_ch - 1])
    assert e["per_ch"] < 1e-4, e


@pytest.mark.parametrize("nx", [2048, 4096])
def test_strang_tmem_form_gives_identical_fields(nx):
    """Strang splitting in the tensor-memory parked form equals the resident form."""
    w = deformed_small(nx, nz=40, n_ch=6, seed=32)
    w.split_order = 2
    ref, _ = fields(w, form=0, channels_per_block=1)
    got, used = fields(w, form=3, channels_per_block=1)
    assert used["form"] == 3
    for k in ("e0", "eh", "R"):
        assert np.array_equal(got[k], ref[k]), k


@pytest.mark.parametrize("nx", [1024, 4096])
def test_fourth_order_parked_form_gives_identical_fields(nx):
    """Fourth-order splitting in the parked form (tables from L2, two sets)
    equals the resident form."""
    w = deformed_small(nx, nz=24, n_ch=5, seed=33)
    w.split_order = 4
    ref, _ = fields(w, form=0, channels_per_block=1)
    got, used = fields(w, form=2, channels_per_block=1)
    assert used["form"] == 2
    for k in ("e0", "eh", "R"):
        assert np.array_equal(got[k], ref[k]), k


@pytest.mark.parametrize("nx,ny,n_ch", [(512, 256, 3), (256, 512, 5), (256, 1024, 2)])
def test_3d_streamed_column_pass_gives_identical_fields(nx, ny, n_ch):
    """Launch form 1 of a 3D plan: the persistent column pass that streams each
    group's next column in with a bulk copy (mbarrier completion) while it
    transforms the current one.  Same arithmetic per element as form 0, so the
    fields are bitwise equal; channel counts leave the last groups short of
    columns (a ragged end of the persistent walk)."""
    from test_gpu_3d import case3d
    w = case3d(nx, ny, 12, n_ch, seed=nx + ny + n_ch)
    a, used_a = fields(w, form=0, row_threads=256)
    b, used_b = fields(w, form=1, row_threads=256)
    assert used_a["form"] == 0 and used_b["form"] == 1
    for k in ("e0", "eh", "R"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("nx,ny,n_ch,rt", [(512, 512, 8, 128), (512, 512, 5, 256),
                                           (256, 512, 9, 128), (1024, 256, 4, 256),
                                           (512, 256, 1, 128)])
def test_3d_streamed_row_pass_gives_identical_fields(nx, ny, n_ch, rt):
    """Launch form 2 of a 3D plan: the MODE-1 row passes stream their tiles in
    and out with tensor copies (swizzled boxes of rt / (nx/16) rows), the next
    tile arriving while the current one is transformed.  Same arithmetic per
    element as form 0, so the fields are bitwise equal.  The channel counts
    give most blocks of the persistent grid two or three tiles (the prefetch
    and the mbarrier phases) with a ragged end; the last case fills only part
    of the grid."""
    from test_gpu_3d import case3d
    w = case3d(nx, ny, 12, n_ch, seed=nx + ny + n_ch + rt)
    a, used_a = fields(w, form=0, row_threads=256)
    b, used_b = fields(w, form=2, row_threads=rt)
    assert used_a["form"] == 0 and used_b["form"] == 2 and used_b["row_threads"] == rt
    for k in ("e0", "eh", "R"):
        assert np.array_equal(a[k], b[k]), k
    p = bpm.plan_from_workload(w)
    with pytest.raises(bpm.BpmError):
        p.set_launch(form=2, row_threads=512)  # no streamed tile of 512 threads
    p.close()


def test_3d_row_tiles_give_identical_fields():
    from test_gpu_3d import case3d
    w = case3d(512, 256, 16, 2, seed=5)
    a, used_a = fields(w, row_threads=256)
    b, used_b = fields(w, row_threads=512)
    assert used_a["row_threads"] == 256 and used_b["row_threads"] == 512
    assert np.array_equal(a["e0"], b["e0"]) and np.array_equal(a["eh"], b["eh"])


def test_forms_a_plan_cannot_run_are_refused():
    w = workloads.tiny(n_ch=4)
    p = bpm.plan_from_workload(w)
    with pytest.raises(bpm.BpmError):
        p.set_launch(row_threads=384)
    with pytest.raises(bpm.BpmError):
        p.set_launch(channels_per_block=3)
    p.close()
    w.split_order = 2
    q = bpm.plan_from_workload(w)
    with pytest.raises(bpm.BpmError):
        q.set_launch(form=1, channels_per_block=16)  # the L2 form is first order only
    with pytest.raises(bpm.BpmError):
        q.set_launch(form=2, channels_per_block=1)   # so is the parked form (and Nx >= 1024)
    with pytest.raises(bpm.BpmError):
        q.set_launch(form=3, channels_per_block=1)   # the TMEM form needs Nx >= 1024
    q.close()
    r = bpm.plan_from_workload(deformed_small(1024, nz=8, n_ch=4, seed=1))
    with pytest.raises(bpm.BpmError):
        r.set_launch(form=3, channels_per_block=1)   # at 1024 it runs two channels a block
    r.set_launch(form=3, channels_per_block=2)
    r.close()


def test_tuner_keeps_the_fastest_and_later_plans_use_it(tmp_path):
    bpm.tune_clear()
    dx = 0.5e-6
    best, every = bpm.tune(2, 1024, 1, dx, 0.0, dx, 611, steps=8)
    assert len(every) == 5 and all(f["ms"] > 0 for f in every)  # smem x2, L2, parked, TMEM
    assert best["ms"] == min(f["ms"] for f in every)
    want = {k: best[k] for k in ("form", "channels_per_block", "row_threads")}
    p = bpm.Plan(2, 1024, 1, 30, dx, 0.0, dx, 611)
    assert p.launch() == want
    p.close()
    path = str(tmp_path / "tune.txt")
    bpm.tune_save(path)
    bpm.tune_clear()
    assert bpm.tune_load(path) == 1
    q = bpm.Plan(2, 1024, 1, 30, dx, 0.0, dx, 611)
    assert q.launch() == want
    q.close()
    b3, every3 = bpm.tune(3, 256, 256, 1e-6, 1e-6, 0.25e-6, 2, steps=4)
    assert {f["row_threads"] for f in every3} == {128, 256, 512}
    assert {f["form"] for f in every3} == {0, 1, 2}
    bpm.tune_clear()
