"""The N > 1 bench path on CPU: two gloo ranks (world size 2, 127.0.0.1).

Default: the ranks split one instance's channels (strong scaling) and
reduce-scatter its time response over t, the one exchange; the value is the
instance's cell-updates over the slowest rank's time.  --independent: ranks
march independent instances (weak scaling, no data-path collective); the only
collective is the MAX of the timed duration, and the reported value is all
ranks' cell-updates over the slowest rank's time."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.rank_workload(n_ch=2, nx=256, nz=8, rank=rank)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
    value = bench.whole_job_value(world, w.cell_updates, ms)
    out[rank] = (ms, float(np.abs(w.u).sum()), value, w.cell_updates)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    (ms0, u0, v0, c0), (ms1, u1, v1, c1) = res[0], res[1]
    assert ms0 == ms1 == 15.0                      # max over ranks
    assert u0 != u1                                # independent instances (seed 2 + rank)
    assert c0 == c1 == 2 * 256 * 8                 # same size per rank (weak scaling)
    assert v0 == v1 == pytest.approx(2 * c0 / 15e-3)


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_value(1, 1000, 2.0) == pytest.approx(5e5)


def _shard_rank(rank, world, port, out):
    """The default N > 1 path's host logic: this rank's channel block of the one
    instance, its part of the time response (the oracle's sum over its block,
    the other channels zero), the reduce-scatter over t, the MAX of the time."""
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle.oracle as orc
    from paper_2201_08500_gb300 import shard
    w, w_all, first = bench.rank_share(n_ch=7, nx=256, nz=8, world=world, rank=rank)
    rng = np.random.default_rng(5)
    eh = rng.normal(size=(w_all.n_ch, 3)) + 1j * rng.normal(size=(w_all.n_ch, 3))
    part = np.zeros_like(eh)
    part[first:first + w.n_ch] = eh[first:first + w.n_ch]
    domega = shard.pulse_spacing(w_all.omega)
    t = torch.from_numpy(orc.omega_to_t(part, domega))
    rows, row0, r_int = shard.combine_scatter(t, float(rank + 1))
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
    out[rank] = (first, w.n_ch, row0, rows.numpy().copy(), r_int, ms,
                 w_all.cell_updates, orc.omega_to_t(eh, domega))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_one_pulse_and_reduce_scatter_its_time_response():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    (f0, c0, r0, rows0, ri0, ms0, cells, full), (f1, c1, r1, rows1, ri1, ms1, _, _) = res[0], res[1]
    assert (f0, c0, f1, c1) == (0, 4, 4, 3)         # contiguous channel blocks of the 7
    assert (r0, rows0.shape[0], r1, rows1.shape[0]) == (0, 4, 4, 3)  # time rows, ceil(7/2)
    got = np.concatenate([rows0, rows1])
    assert np.max(np.abs(got - full)) <= 1e-12 * np.max(np.abs(full))
    assert ri0 == ri1 == 3.0                        # R_int parts summed
    assert ms0 == ms1 == 15.0
    assert cells == 7 * 256 * 8                     # strong scaling: the one instance's work
