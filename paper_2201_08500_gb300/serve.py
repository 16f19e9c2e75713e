"""Continuous-batching BPM server on one GPU (driver of the C++ batch executor).

Requests are workload records (one crystal + pulse each) with arrival times.
The served form:
  * admits a request when a plan slot of its shape is free, or when the device
    memory budget allows a new slot (plans are pooled by shape, so the steady
    state allocates nothing);
  * sets its crystal and pulse on a setup stream (fields stay on the device);
  * advances every admitted request by rounds of `chunk` z steps, each round
    one persistent work-queue launch; requests admitted while earlier ones are
    on the GPU join the next round, and slots free as requests complete;
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


class Server:
    """Continuous batching over a bpm.Batch with plan slots pooled by shape."""

    def __init__(self, hbm_budget_bytes: int, chunk: int = 256, stream=None, keep_fields=True):
        import torch
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.setup_stream = torch.cuda.Stream()
        self.budget = int(hbm_budget_bytes)
        self.chunk = int(chunk)
        self.batch = bpm.Batch(hbm_budget_bytes=0, stream=self.stream)
        self.pool = collections.defaultdict(list)  # shape -> free plans
        self.bytes_in_slots = 0
        self.keep_fields = keep_fields
        self.n_slots = 0

    def _slot(self, w):
        free = self.pool[shape_key(w)]
        if free:
            return free.pop()
        need = bpm.plan_bytes(w.dims, w.nx, w.ny, w.nz, w.n_ch, host_u=w.u is not None)
        if self.bytes_in_slots + need > self.budget:
            return None
        p = bpm.Plan(w.dims, w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.n_ch,
                     stream=self.setup_stream, zassenhaus=w.zassenhaus)
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
        active = {}   # ticket -> (req, plan, steps still to enqueue)
        t0 = time.perf_counter()
        rounds = 0
        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while waiting:
                req = waiting[0]
                p = self._slot(req.work)
                if p is None:
                    break  # no memory for a new slot of this shape yet
                self._load(p, req)
                t = self.batch.submit(p)
                active[t] = [req, p, req.work.nz]
                waiting.popleft()
            todo = [a for a in active.values() if a[2] > 0]
            if todo:
                self.batch.step(self.chunk)
                rounds += 1
                for a in todo:
                    a[2] = max(0, a[2] - self.chunk)
            else:
                time.sleep(5e-5)
            for t in list(active):
                if self.batch.poll(t):
                    req, p, _ = active.pop(t)
                    req.R = p.reflectivity()[0]
                    if self.keep_fields:
                        req.eh = p.eh()
                    req.done_at = time.perf_counter() - t0
                    self.pool[shape_key(req.work)].append(p)
            if not todo and not waiting and pending and not active:
                dt = pending[0].arrival - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(min(dt, 0.01))
        self.rounds = rounds
        return requests

    def close(self):
        for plans in self.pool.values():
            for p in plans:
                p.close()
        self.pool.clear()
        self.batch.close()


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


def summarize(requests) -> dict:
    lat = np.array([r.done_at - r.arrival for r in requests])
    cells = sum(r.work.cell_updates for r in requests)
    span = max(r.done_at for r in requests) - min(r.arrival for r in requests)
    return {"requests": len(requests), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "makespan_s": float(span), "cell_updates": int(cells),
            "throughput": float(cells / span)}
