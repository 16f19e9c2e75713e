"""Frequency sharding of one pulse across ranks, one GPU each.

Section 3.3 solves every frequency component of the pulse as an independent
stationary problem. Only two sums combine the channels: the time response
psi_h(t_j, x) (Section 3.3) and the integrated reflectivity R_int
(Section 3.1). So a pulse shards by channel:
- each rank marches a contiguous block of channels in its own plan;
- bpm_set_channel_shard makes that plan's time response and R_int this
  block's parts of the two sums, with the global channel indices in the phase
  factors;
- one sum-reduce over the process group combines the parts: combine()
  leaves the whole sum on every rank (an all-reduce), combine_scatter() a
  block of time rows on each (a reduce-scatter over t, half the traffic).

The per-channel R_i need no reduce: each rank holds its own block's values.
"""
from __future__ import annotations

import numpy as np

from . import bpm


def channel_blocks(n_total: int, world: int) -> list[tuple[int, int]]:
    """Contiguous (first, count) per rank. Counts differ by at most one, and
    the first n_total % world ranks take the larger count."""
    if n_total < 1 or world < 1:
        raise ValueError("n_total and world must be >= 1")
    base, extra = divmod(n_total, world)
    out, first = [], 0
    for r in range(world):
        cnt = base + (1 if r < extra else 0)
        out.append((first, cnt))
        first += cnt
    return out


def pulse_spacing(omega) -> float:
    """Channel spacing of the whole pulse (1 for a single channel, as a plan uses)."""
    omega = np.asarray(omega, np.float64)
    return float(omega[1] - omega[0]) if omega.size > 1 else 1.0


def combine(time_part, r_int_part: float, group=None):
    """Sum-reduce a shard's time response (a torch tensor, complex128, on the
    device of the group's backend) in place, and the shard's R_int; returns
    the pulse's R_int.  A process group of one rank (or none) is the identity."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(r_int_part)
    dist.all_reduce(torch.view_as_real(time_part), op=dist.ReduceOp.SUM, group=group)
    r = torch.tensor([float(r_int_part)], dtype=torch.float64, device=time_part.device)
    dist.all_reduce(r, op=dist.ReduceOp.SUM, group=group)
    return float(r.item())


def time_row_blocks(n_time: int, world: int) -> list[tuple[int, int]]:
    """Rows of the time response each rank holds after combine_scatter: equal
    blocks of ceil(n_time / world) rows (the last ones shorter or empty)."""
    if n_time < 1 or world < 1:
        raise ValueError("n_time and world must be >= 1")
    per = -(-n_time // world)
    return [(min(r * per, n_time), max(0, min(per, n_time - r * per))) for r in range(world)]


def combine_scatter(time_part, r_int_part: float, group=None):
    """Reduce-scatter a shard's time response over t: every rank sends its
    part of the whole [n_time, plane] sum and keeps the sum of its own block of
    time rows (time_row_blocks), half the traffic of an all-reduce.  Returns
    (rows, first_row, R_int): rows is this rank's block [count, plane] of the
    pulse's time response (complex128, on time_part's device) and R_int the
    pulse's.  A process group of one rank (or none) returns time_part whole."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return time_part, 0, float(r_int_part)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n_time, plane = time_part.shape
    per = -(-n_time // world)
    flat = torch.view_as_real(time_part).reshape(-1)
    if per * world != n_time:
        pad = torch.zeros((per * world - n_time) * plane * 2, dtype=flat.dtype, device=flat.device)
        flat = torch.cat([flat, pad])
    out = torch.empty(per * plane * 2, dtype=flat.dtype, device=flat.device)
    dist.reduce_scatter_tensor(out, flat, op=dist.ReduceOp.SUM, group=group)
    first, cnt = time_row_blocks(n_time, world)[rank]
    rows = torch.view_as_complex(out.view(per, plane, 2))[:cnt]
    r = torch.tensor([float(r_int_part)], dtype=torch.float64, device=time_part.device)
    dist.all_reduce(r, op=dist.ReduceOp.SUM, group=group)
    return rows, first, float(r.item())


def shard_plan(w, rank: int, world: int, stream=None):
    """The plan of rank's channel block of workload w (None when the block is
    empty, i.e. more ranks than channels), set up and sharded but not run."""
    first, cnt = channel_blocks(w.n_ch, world)[rank]
    if cnt == 0:
        return None, first, cnt
    p = bpm.plan_from_workload(w.subset(list(range(first, first + cnt))), stream=stream)
    p.set_channel_shard(first, w.n_ch, pulse_spacing(w.omega))
    return p, first, cnt


def run_sharded(w, rank: int = 0, world: int = 1, group=None, stream=None) -> dict:
    """March rank's channel block of workload w on the current GPU and combine
    the time response and R_int over the group.

    Returns time (complex128 [n_ch, plane] on the GPU, the whole pulse's after
    the reduce), R_int (the pulse's), R (this block's channels) and the block's
    first and count."""
    import torch
    p, first, cnt = shard_plan(w, rank, world, stream=stream)
    t = torch.zeros((w.n_ch, w.plane), dtype=torch.complex128, device="cuda")
    R = np.empty(0)
    r_int = 0.0
    if p is not None:
        p.run()
        p.sync()
        R, _, r_int = p.reflectivity()
        p.fetch(bpm.BPM_FIELD_EH_TIME, out=t)
        p.close()
    r_int = combine(t, r_int, group=group)
    return dict(time=t, R_int=r_int, R=R, first=first, count=cnt)
