"""Channel shards of one pulse (bpm_set_channel_shard) on the GPU: the shards'
time responses and R_int add up to those of one plan holding every channel,
and their per-channel R are that plan's (Section 3.3: channels are
independent; the time response and R_int are the only sums over them)."""
import numpy as np
import pytest
import torch

from paper_2201_08500_gb300 import bpm, shard, workloads
from test_gpu_parity import deformed_small

pytestmark = pytest.mark.gpu


def whole(w):
    p = bpm.plan_from_workload(w)
    p.run()
    p.sync()
    R, _, r_int = p.reflectivity()
    t = p.eh_time()
    p.close()
    return t, R, r_int


def shards(w, world):
    t = np.zeros((w.n_ch, w.plane), np.complex128)
    R, r_int = [], 0.0
    for rank in range(world):
        p, first, cnt = shard.shard_plan(w, rank, world)
        if p is None:
            continue
        p.run()
        p.sync()
        Rp, _, rp = p.reflectivity()
        tp = p.eh_time()
        assert tp.shape == (w.n_ch, w.plane)
        t += tp
        R.append(Rp)
        r_int += rp
        p.close()
    return t, np.concatenate(R), r_int


@pytest.mark.parametrize("n_ch,world", [(8, 3), (6, 4), (5, 8)])
def test_channel_shards_add_up_to_the_whole_pulse(n_ch, world):
    # 8 channels: power-of-two transform kernel; 6 and 5: direct sum; 5 over 8
    # ranks leaves three ranks without channels
    w = deformed_small(1024, nz=60, n_ch=n_ch, seed=11)
    t_all, R_all, rint_all = whole(w)
    t_sh, R_sh, rint_sh = shards(w, world)
    assert np.array_equal(R_sh, R_all)                    # channel independence
    assert np.max(np.abs(t_sh - t_all)) <= 1e-12 * np.max(np.abs(t_all))
    assert rint_sh == pytest.approx(rint_all, rel=1e-12)


def test_3d_channel_shards_add_up_to_the_whole_pulse():
    from test_gpu_3d import case3d
    w = case3d(256, 256, 6, 4, seed=12)
    t_all, R_all, rint_all = whole(w)
    t_sh, R_sh, rint_sh = shards(w, 2)
    assert np.array_equal(R_sh, R_all)
    assert np.max(np.abs(t_sh - t_all)) <= 1e-12 * np.max(np.abs(t_all))
    assert rint_sh == pytest.approx(rint_all, rel=1e-12)


def test_run_sharded_on_one_rank_is_the_whole_pulse():
    w = deformed_small(1024, nz=40, n_ch=4, seed=13)
    t_all, R_all, rint_all = whole(w)
    out = shard.run_sharded(w)
    assert out["first"] == 0 and out["count"] == w.n_ch
    assert np.array_equal(out["R"], R_all)
    assert np.array_equal(out["time"].cpu().numpy(), t_all)
    assert out["R_int"] == rint_all


def test_channel_shard_arguments_are_checked():
    w = workloads.tiny(n_ch=4)
    p = bpm.plan_from_workload(w)
    for bad in [(-1, 8, 1.0), (6, 8, 1.0), (0, 3, 1.0), (0, 8, 0.0), (0, 8, float("nan"))]:
        with pytest.raises(bpm.BpmError):
            p.set_channel_shard(*bad)
    p.run(3)
    with pytest.raises(bpm.BpmError):
        p.set_channel_shard(0, 8, 1.0)                    # the march has started
    p.close()
    q = bpm.plan_from_workload(w)
    q.set_channel_shard(2, 8, 1.0)
    q.run()
    q.sync()
    out = torch.empty((8, w.plane), dtype=torch.complex128, device="cuda")
    q.fetch(bpm.BPM_FIELD_EH_TIME, out=out)               # n_total rows, on the device
    with pytest.raises(bpm.BpmError):
        q.fetch(bpm.BPM_FIELD_EH_TIME, out=np.empty((4, w.plane), np.complex128))
    q.close()
