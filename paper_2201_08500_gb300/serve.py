"""Continuous-batching BPM server on one GPU (the host loop over the C++ batch executor).

Requests are workload records (one crystal + pulse each) with arrival times.
The served form:
  * admits a request when a plan slot of its shape is free, or when the device
    memory budget allows a new slot (plans are pooled by shape, so the steady
    state allocates nothing);
  * sends it to one of two lanes by size: short requests (single-channel
    probes) to a lane on a few reserved SMs, the rest to a lane on the others;
  * sets its crystal and pulse on the lane's setup stream (fields stay on the
    device);
  * advances every admitted request by rounds (long lane: `chunk` z steps;
    short lane: to completion), each round one persistent work-queue launch
    per queue; requests admitted while earlier ones are on the GPU join the
    next round, and slots free as requests complete;
  * on completion copies the result (reflectivities and the reflected field)
    to the host and returns the slot.
The plain form serves the same arrivals one request at a time with one march
launch per request.  Both report p50 / p99 latency (completion - arrival) and
throughput in cell-updates per second over the makespan.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import bpm


@dataclasses.dataclass
class Request:
    rid: int
    work: object          # workload record
    u_dev: object         # device displacement (torch tensor) or None
    arrival: float        # seconds after the start of the run
    done_at: float = -1.0
    R: np.ndarray | None = None
    eh: np.ndarray | None = None


def shape_key(w):
    return (w.nx, w.nz, w.n_ch, w.dx, w.dz, w.zassenhaus)


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


class _Lane:
    """One batch with its own stream, setup stream, SM cap and round length."""

    def __init__(self, torch, max_blocks: int, chunk: int, stream=None, priority: int = 0):
        self.stream = stream if stream is not None else torch.cuda.Stream(priority=priority)
        self.setup_stream = torch.cuda.Stream()
        self.batch = bpm.Batch(hbm_budget_bytes=0, stream=self.stream)
        if max_blocks > 0:
            self.batch.set_max_blocks(max_blocks)
        self.chunk = int(chunk)
        self.active = {}   # ticket -> [req, plan, steps still to enqueue]
        self.rounds = 0


class Server:
    """Continuous batching over bpm.Batch lanes with plan slots pooled by shape.

    Requests of at most `short_cells` cell-updates (single-channel probes) go to
    a short lane that owns `short_sms` SMs and runs each request to completion in
    one round; everything else goes to the long lane (the other SMs, rounds of
    `chunk` steps).  The persistent launches of the two lanes hold one block per
    SM, so their blocks fit side by side and a probe does not wait behind a long
    round; the short lane's stream has the higher priority, so that its blocks
    are placed first when SMs free up.  short_sms = 0 gives one lane on every SM.
    """

    def __init__(self, hbm_budget_bytes: int, chunk: int = 256, stream=None, keep_fields=True,
                 short_cells: float = 1e7, short_sms: int = 4):
        import torch
        self.torch = torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        self.budget = int(hbm_budget_bytes)
        self.short_cells = float(short_cells) if short_sms > 0 else -1.0
        self.long = _Lane(torch, sms - short_sms if short_sms > 0 else 0, chunk,
                          stream if stream is not None else torch.cuda.current_stream())
        # high priority: when a long kernel's blocks retire, waiting probe blocks go first
        self.short = _Lane(torch, short_sms, 1 << 30, priority=-1) if short_sms > 0 else None
        self.pool = collections.defaultdict(list)  # shape -> free plans
        self.bytes_in_slots = 0
        self.keep_fields = keep_fields
        self.n_slots = 0

    @property
    def rounds(self):
        return self.long.rounds + (self.short.rounds if self.short else 0)

    def _lane(self, w):
        return self.short if w.cell_updates <= self.short_cells else self.long

    def _slot(self, w, lane):
        free = self.pool[shape_key(w)]
        if free:
            return free.pop()
        need = bpm.plan_bytes(w.dims, w.nx, w.ny, w.nz, w.n_ch, host_u=w.u is not None)
        if self.bytes_in_slots + need > self.budget:
            return None
        p = bpm.Plan(w.dims, w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.n_ch,
                     stream=lane.setup_stream, zassenhaus=w.zassenhaus)
        p.bytes = need
        self.bytes_in_slots += need
        self.n_slots += 1
        return p

    def _load(self, p, req):
        w = req.work
        p.set_crystal(w.chi0, w.chih, w.chihb, w.theta_B, w.lambda_B, w.x_surface, w.thickness,
                      u=req.u_dev if req.u_dev is not None else w.u)
        p.set_pulse(w.omega, w.S, w.theta_i, w.x0, w.w0, w.zx, w.zR)

    def serve(self, requests):
        """Run the arrival process in real time; fills done_at, R (and eh)."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        lanes = [lane for lane in (self.short, self.long) if lane is not None]
        t0 = time.perf_counter()
        while pending or waiting or any(lane.active for lane in lanes):
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            blocked = collections.deque()
            while waiting:
                req = waiting.popleft()
                lane = self._lane(req.work)
                p = self._slot(req.work, lane)
                if p is None:
                    blocked.append(req)  # no memory for a new slot of this shape yet
                    continue
                self._load(p, req)
                t = lane.batch.submit(p)
                lane.active[t] = [req, p, req.work.nz]
            waiting = blocked
            stepped = False
            for lane in lanes:
                todo = [a for a in lane.active.values() if a[2] > 0]
                # keep at most two rounds in flight so that a step never blocks
                if todo and lane.batch.pending() < 2:
                    lane.batch.step(lane.chunk)
                    lane.rounds += 1
                    stepped = True
                    for a in todo:
                        a[2] = max(0, a[2] - lane.chunk)
            for lane in lanes:
                for t in list(lane.active):
                    if lane.batch.poll(t):
                        req, p, _ = lane.active.pop(t)
                        req.R = p.reflectivity()[0]
                        if self.keep_fields:
                            req.eh = p.eh()
                        req.done_at = time.perf_counter() - t0
                        self.pool[shape_key(req.work)].append(p)
            if not stepped:
                idle = not waiting and not any(lane.active for lane in lanes)
                dt = pending[0].arrival - (time.perf_counter() - t0) if (idle and pending) else 5e-5
                if dt > 0:
                    time.sleep(min(dt, 0.01))
        return requests

    def close(self):
        for plans in self.pool.values():
            for p in plans:
                p.close()
        self.pool.clear()
        for lane in (self.short, self.long):
            if lane is not None:
                lane.batch.close()


def serve_plain(requests, stream=None, keep_fields=True):
    """One request at a time, FIFO, one march launch per request (plans cached
    by shape so that this form, too, allocates nothing in the steady state)."""
    import torch
    stream = stream if stream is not None else torch.cuda.current_stream()
    cache = {}
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if req.arrival > now:
            time.sleep(req.arrival - now)
        w = req.work
        key = shape_key(w)
        if key not in cache:
            cache[key] = bpm.Plan(w.dims, w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.n_ch,
                                  stream=stream, zassenhaus=w.zassenhaus)
        p = cache[key]
        p.set_crystal(w.chi0, w.chih, w.chihb, w.theta_B, w.lambda_B, w.x_surface, w.thickness,
                      u=req.u_dev if req.u_dev is not None else w.u)
        p.set_pulse(w.omega, w.S, w.theta_i, w.x0, w.w0, w.zx, w.zR)
        p.run()
        req.R = p.reflectivity()[0]
        if keep_fields:
            req.eh = p.eh()
        req.done_at = time.perf_counter() - t0
    for p in cache.values():
        p.close()
    return requests


def summarize(requests, short_cells: float = 1e7) -> dict:
    """Latency percentiles (all requests, and short / long ones apart) and
    throughput in cell-updates per second over the makespan."""
    def pct(rs):
        if not rs:
            return {}
        lat = np.array([r.done_at - r.arrival for r in rs]) * 1e3
        return {"n": len(rs), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean())}

    cells = sum(r.work.cell_updates for r in requests)
    span = max(r.done_at for r in requests) - min(r.arrival for r in requests)
    out = pct(requests)
    out["requests"] = out.pop("n")
    out.update({"makespan_s": float(span), "cell_updates": int(cells),
                "throughput": float(cells / span),
                "short": pct([r for r in requests if r.work.cell_updates <= short_cells]),
                "long": pct([r for r in requests if r.work.cell_updates > short_cells])})
    return out
