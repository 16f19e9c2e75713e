"""Frequency sharding of one pulse across ranks, host side on CPU: three gloo
ranks (127.0.0.1) each hold a channel block's part of the time response, and
one sum-reduce (an all-reduce, or a reduce-scatter over t) gives the whole
pulse's (Section 3.3: the channels are
independent; the time response and R_int are the only sums over them)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2201_08500_gb300 import shard  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_channel_blocks_partition_the_pulse():
    for n in (1, 2, 7, 8, 1024):
        for world in (1, 2, 3, 8, 11):
            blocks = shard.channel_blocks(n, world)
            assert len(blocks) == world
            assert blocks[0][0] == 0
            for (f0, c0), (f1, _) in zip(blocks, blocks[1:]):
                assert f1 == f0 + c0                      # contiguous
            assert sum(c for _, c in blocks) == n         # covers every channel once
            counts = [c for _, c in blocks]
            assert max(counts) - min(counts) <= 1
            assert counts == sorted(counts, reverse=True)
    with pytest.raises(ValueError):
        shard.channel_blocks(0, 2)


def _spectrum(n, plane, seed=21):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(n, plane)) + 1j * rng.normal(size=(n, plane))).astype(np.complex64)


def _rank(rank, world, port, n, plane, domega, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle.oracle as orc
    from paper_2201_08500_gb300 import shard as sh
    eh = _spectrum(n, plane)
    first, cnt = sh.channel_blocks(n, world)[rank]
    part = np.zeros_like(eh)
    part[first:first + cnt] = eh[first:first + cnt]       # the other ranks' channels count as zero
    t = torch.from_numpy(orc.omega_to_t(part.astype(np.complex128), domega))
    R = np.linspace(0.1, 0.9, n)                          # stand-in per-channel reflectivities
    t2 = torch.from_numpy(orc.omega_to_t(part.astype(np.complex128), domega))
    rows, row0, r_int2 = sh.combine_scatter(t2, domega * float(R[first:first + cnt].sum()))
    r_int = sh.combine(t, domega * float(R[first:first + cnt].sum()))
    out[rank] = (t.numpy(), r_int, rows.numpy().copy(), row0, r_int2)
    dist.barrier()
    dist.destroy_process_group()


def test_three_gloo_ranks_sum_their_parts_to_the_whole_time_response():
    import torch.multiprocessing as mp
    import oracle.oracle as orc
    n, plane, domega = 8, 5, 2.5e12
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 3, port, n, plane, domega, out))
                 for r in range(3)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        res = dict(out)
    full = orc.omega_to_t(_spectrum(n, plane).astype(np.complex128), domega)
    for r in range(3):
        t, r_int, _, _, r_int2 = res[r]
        assert np.max(np.abs(t - full)) <= 1e-12 * np.max(np.abs(full))
        assert r_int == pytest.approx(domega * np.linspace(0.1, 0.9, n).sum(), rel=1e-14)
        assert r_int2 == pytest.approx(r_int, rel=1e-14)
    # reduce-scatter over t: blocks of ceil(8 / 3) = 3 rows, the last one shorter
    assert [(res[r][3], res[r][2].shape[0]) for r in range(3)] == shard.time_row_blocks(n, 3) \
        == [(0, 3), (3, 3), (6, 2)]
    got = np.concatenate([res[r][2] for r in range(3)])
    assert np.max(np.abs(got - full)) <= 1e-12 * np.max(np.abs(full))


def test_a_shard_part_carries_the_global_channel_phase():
    """One channel at global index i0 of n, amplitude A: its part of the time
    response is d_omega A exp(-2 pi i (i0 - n/2) j / n) (closed form)."""
    import oracle.oracle as orc
    n, i0, A, domega = 8, 5, 0.3 - 0.7j, 1.5
    part = np.zeros((n, 1), np.complex128)
    part[i0, 0] = A
    t = orc.omega_to_t(part, domega)[:, 0]
    j = np.arange(n)
    want = domega * A * np.exp(-2j * np.pi * (i0 - n // 2) * j / n)
    assert np.max(np.abs(t - want)) < 1e-15 * n


def test_single_rank_combine_is_the_identity():
    import torch
    t = torch.ones(3, 2, dtype=torch.complex128)
    assert shard.combine(t, 4.5) == 4.5
    assert torch.equal(t, torch.ones(3, 2, dtype=torch.complex128))
