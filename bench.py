"""Benchmark of the two-beam FFT BPM hot path on GB300.

A step is one pass of the whole hot path over one synthetic workload: the
deformation factor c(x, z) from the displacement field, the per-channel
propagator tables and coupling coefficients, the incident field, the resident
split-step march of every channel, the reflectivities and the frequency-to-time
assembly.  Default workload: deformed crystal, Nx = 4096, 2000 z steps, 1024
frequency channels (8.39e9 cell-updates per step).  The metric is
cell-updates per second (channel x transverse cell x z step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

At N = 1 the one JSON line also carries, as nested objects, the other
workloads of the method: `batched` (64 uneven instances in one CUDA graph of
persistent work-queue launches against one launch per instance), `served` (a
Poisson stream of 10,000 requests served with continuous batching against
plain per-request launches, p50/p99 latency) and `3d` (512 x 512 transverse,
1000 steps, 128 channels, HBM-streamed, against the HBM roofline).  Each has
its own clock record and a parity sample against the FP64 oracle; the oracle
samples run on the host in a background thread while the GPU goes on.
--no-extras skips them.  `peaks` holds the measured FP32 and FP64 CUDA-core
rates (FMA chains on every SM) that the ALU rooflines divide by.

N > 1 runs under torchrun: the ranks split ONE instance's channels into
contiguous blocks (strong scaling) and reduce-scatter its time response over
t, the one exchange of a sharded pulse.  --independent instead marches one
instance per rank (weak scaling, no data-path collective).  --impl reference
times the FP64 CPU oracle on the host cores on a bounded channel sample.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2201_08500_gb300 import workloads  # noqa: E402

METRIC = "BPM cell-updates/s (omega*x*z)"
UNIT = "cell-updates/s"
FP32_LANES_PER_SM = 128
TOL_FIELD = 1e-4

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# default march, from one ncu capture of that launch (form 3 with the packed
# FP32 butterflies: 555.43 MB read + 55.04 MB written).  The deformation rows
# are re-read by each wave of channels, which at ~10 GB/s is immaterial to this
# ALU-bound kernel.  Keyed by kernel, form and workload; any other
# configuration (or a kernel changed since the capture) reports null.
MEASURED_TRAFFIC = {
    ("march_kernel<4096,1> form 3", "deformed-2d-nx4096-nz2000-ch1024", 1): 610.46e6,
}
# Executed FP32 flop per cell-update (FADD + FMUL + 2 FFMA thread instructions,
# ncu, per kernel and form): the work the kernel really issues, against the
# nominal count of flops_per_cell.  Counted on the build with scalar
# butterfly additions; the packed build performs the same operations (its
# fields are bitwise equal at these sizes), and ncu's per-opcode FP32 counters
# do not resolve the packed two-lane instructions.  8192: 240 counted, less
# the products by one that the lane-pair twiddles dropped since (7 complex
# products of 6 flop per thread, four times a step, over 16 cell-updates).
EXECUTED_FLOPS = {
    "march_kernel<4096,1> form 3": 210.0,
    "march_kernel<8192,1> form 3": 240.0 - 7 * 6 * 4 / 16,
}
# DRAM bytes of one z step of the 3D workload (one streamed column pass, launch
# form 1, + one MODE-1 row pass, 256-thread row tile), from the live launch
# list of those launches with --cache-control none: 1066.2 + 1082.6 MB, the
# algorithmic 64 B per cell-update (2147 MB) within 0.1 %.
MEASURED_TRAFFIC_3D = {("large-3d-512x512-nz1000-ch128", 1, 256): (539.6e6 + 526.6e6 + 537.6e6
                                                                     + 545.0e6),
                       ("large-3d-512x512-nz1000-ch128", 2, 128): (539.5e6 + 528.3e6 + 538.5e6
                                                                     + 544.5e6)}


def flops_per_cell(n: int, split_order: int = 1) -> float:
    """Nominal FLOPs per cell-update: per propagation 4 FFTs at 5 N log2 N (20
    log2 N per cell) and 2 propagator multiplies (12), per coupling 40.
    Eq. split-op: order 1 has 1 propagation and 1 coupling, order 2 one and
    two, order 4 three and four."""
    props, couplings = {1: (1, 1), 2: (1, 2), 4: (3, 4)}[split_order]
    return props * (20.0 * math.log2(n) + 12.0) + couplings * 40.0


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The slowest rank's time (an all-reduce MAX of one number; identity at N = 1)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, cells_per_rank: int, ms: float) -> float:
    """Cell-updates of all ranks divided by the slowest rank's time."""
    return world * cells_per_rank / (ms * 1e-3)


def rank_workload(n_ch: int, nx: int, nz: int, rank: int):
    """--independent: each rank marches its own instance of the same size
    (seed 2 + rank); channels and instances are independent, so ranks exchange
    no data."""
    return workloads.deformed(n_ch=n_ch, nx=nx, nz=nz, seed=2 + rank)


def rank_share(n_ch: int, nx: int, nz: int, world: int, rank: int):
    """Default at N > 1: the ranks split ONE instance (seed 2) into contiguous
    channel blocks.  Returns (this rank's workload, the whole instance, its
    first channel); the job's work is the whole instance's cell-updates."""
    from paper_2201_08500_gb300 import shard
    w_all = workloads.deformed(n_ch=n_ch, nx=nx, nz=nz, seed=2)
    first, cnt = shard.channel_blocks(w_all.n_ch, world)[rank]
    if cnt == 0:
        raise SystemExit("a sharded pulse needs at least one channel per rank")
    return w_all.subset(list(range(first, first + cnt))), w_all, first


# --------------------------------------------------------------------------- oracle legs
def oracle_sample(w, n_channels: int, n_threads: int, keep: bool = False):
    """Time the FP64 oracle (as it stands) on n_channels channels of workload w
    spread over the band; keep=True also returns (channel indices, e0, eh, init)."""
    import oracle.oracle as orc
    orc.build()
    idx = np.linspace(0, w.n_ch - 1, n_channels).round().astype(int)
    t0 = time.perf_counter()
    out = orc.run(w, channels=idx, n_threads=n_threads)
    dt = time.perf_counter() - t0
    cells = n_channels * w.plane * w.nz
    if keep:
        return cells / dt, dt, cells, (idx,) + tuple(out)
    return cells / dt, dt, cells


def field_errors(w, channels, g0, gh, n_threads):
    """GPU fields g0, gh ([len(channels), plane], the final z) of channels of
    workload w against the oracle: per-channel error relative to the incident
    field's norm, rel-L2 of each field, and R_i."""
    import oracle.oracle as orc
    o0, oh, init = orc.run(w, channels=channels, n_threads=n_threads)
    g0 = np.asarray(g0).reshape(len(channels), -1)
    gh = np.asarray(gh).reshape(len(channels), -1)
    return parity_figures(g0, gh, o0, oh, init), orc.reflectivity(init, o0, oh)[0]


def parity_figures(g0, gh, o0, oh, init) -> dict:
    """Error figures of GPU fields against the oracle's.  The bar (1e-4) is on
    the per-channel error relative to the incident field's norm (the scheme is
    linear in the incident field) and on the rel-L2 of the fields.  rel_l2_fields
    takes both envelopes together (their total power is fixed by the incident
    field); rel_l2_eh is the reflected field alone.  A nearly extinguished E0
    (a perfect crystal's transmitted beam inside the reflection band) makes
    E0's own rel-L2 ill-conditioned, so it is not a bar."""
    inc = np.linalg.norm(init, axis=1)
    err = np.maximum(np.linalg.norm(g0 - o0, axis=1), np.linalg.norm(gh - oh, axis=1)) / inc
    dd = np.sqrt(np.linalg.norm(g0 - o0) ** 2 + np.linalg.norm(gh - oh) ** 2)
    nn = np.sqrt(np.linalg.norm(o0) ** 2 + np.linalg.norm(oh) ** 2)
    return dict(max_err_per_channel=float(err.max()), median_err_per_channel=float(np.median(err)),
                rel_l2_fields=float(dd / nn),
                rel_l2_eh=float(np.linalg.norm(gh - oh) / np.linalg.norm(oh)))


class OracleJobs:
    """Parity samples against the FP64 oracle, run one after another in a
    background thread (the oracle's C march releases the GIL) while the GPU
    sections go on; `threads` host threads each."""

    def __init__(self, threads: int):
        self.threads = max(1, threads)
        self.pool = cf.ThreadPoolExecutor(max_workers=1)
        self.jobs = {}

    def submit(self, name, fn, *args):
        self.jobs[name] = (time.perf_counter(), self.pool.submit(fn, *args))

    def result(self, name):
        t0, fut = self.jobs[name]
        try:
            out = fut.result()
        except Exception as e:  # reported in the line, never silently dropped
            out = {"error": repr(e)[:300]}
        return out

    def close(self):
        self.pool.shutdown(wait=True)


def run_reference(args, world, rank):
    """The FP64 oracle as it stands, on the host cores: each step is one bounded
    sample of the workload (2 channels per core, spread over the band, full
    march).  ms_per_step is the sample's own time; value is the sample's
    cell-updates per second."""
    if rank != 0:
        return 0
    w = workloads.deformed(n_ch=args.channels, nx=args.nx, nz=args.nz)
    cores = os.cpu_count() or 1
    n = max(1, min(w.n_ch, 2 * cores))
    for _ in range(args.warmup):
        oracle_sample(w.subset(range(0, w.n_ch, max(1, w.n_ch // n))), 1, 1)
    vals, dts = [], []
    for _ in range(args.steps):
        v, dt, cells = oracle_sample(w, n, cores)
        vals.append(v)
        dts.append(dt)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(dts), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "nz": w.nz, "channels": w.n_ch,
                   "l2": "n/a (CPU)",
                   "step": f"one sample of {n} of the {w.n_ch} channels (full {w.nz}-step "
                           f"march each); ms_per_step is the sample's time"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} of {w.n_ch} channels, full {w.nz}-step march, "
                                   f"per step; throughput per cell-update of the sample"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- measured peaks
def measure_cuda_core_peaks(local: int) -> dict:
    """FP32 (FFMA) and FP64 (DFMA) chains on every SM (bpm_measure_peak): each
    launch sized to ~150 ms, median of 5, SM clock sampled during them."""
    import torch
    from paper_2201_08500_gb300 import bpm
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    out = {}
    for kind, name, iters in ((bpm.BPM_PEAK_FP32, "fp32", 1 << 18),
                              (bpm.BPM_PEAK_FP64, "fp64", 1 << 12)):
        bpm.measure_peak(kind, max(1, iters // 16))
        _, ms = bpm.measure_peak(kind, iters)
        iters = max(1, int(iters * 150.0 / max(ms, 1e-3)))
        sampler = ClockSampler(local).start()
        runs = [bpm.measure_peak(kind, iters) for _ in range(5)]
        clocks = sampler.stop()
        rate = statistics.median(r for r, _ in runs)
        mhz = clocks.get("sm_mhz") or measured_peaks().get("sm_max_mhz", 2070.0)
        out[name] = {"tflops": rate / 1e12, "launch_ms": statistics.median(m for _, m in runs),
                     "flop_per_clock_per_sm": rate / (sms * mhz * 1e6), "clocks": clocks,
                     "how": "independent FMA chains, 1024 threads per SM (bpm_measure_peak)"}
    return out


# --------------------------------------------------------------------------- config 3
def run_batched(args, world, rank, local, jobs=None):
    """Uneven batch: every instance's full hot path (setup, march, time response),
    once as one CUDA graph around the work-queue launches, once as one march
    launch per instance (the plain form), on the same plans.  Returns the
    `batched` object; with jobs, sampled channels go to the oracle."""
    import torch
    from paper_2201_08500_gb300 import bpm

    torch.cuda.set_device(local)
    ws = workloads.batch(n_inst=args.instances, seed=3 + rank)
    stream = torch.cuda.current_stream()
    us = [None if w.u is None else torch.from_numpy(np.ascontiguousarray(w.u)).cuda() for w in ws]
    # the plain form runs each instance in the launch form the autotuner picks
    # for its shape (untimed setup)
    tuned = {}
    for w in ws:
        key = (w.nx, w.n_ch)
        if key not in tuned:
            tuned[key] = bpm.tune(w.dims, w.nx, w.ny, w.dx, w.dy, w.dz, w.n_ch, steps=256)[0]
    plans = [bpm.plan_from_workload(w, stream=stream, u=u) for w, u in zip(ws, us)]
    cells = sum(w.cell_updates for w in ws)
    b = bpm.Batch(stream=stream)
    for p in plans:
        b.submit(p)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def plain_step():
        for w, p, u in zip(ws, plans, us):
            p.set_crystal(w.chi0, w.chih, w.chihb, w.theta_B, w.lambda_B, w.x_surface,
                          w.thickness, u=u)
            p.set_pulse(w.omega, w.S, w.theta_i, w.x0, w.w0, w.zx, w.zR)
            p.run()

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        out = []
        for i in range(steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    steps_b = max(3, min(args.steps, args.extra_steps))
    sampler = ClockSampler(local).start()
    ms_batched = timed(b.run_graph, steps_b, 3)
    clocks = sampler.stop()
    # parity sample: per transform size the instance with the most z steps,
    # its first, middle and last channel (fields of the last graph pass)
    picks = []
    for nx in sorted({w.nx for w in ws}):
        i = max((k for k, w in enumerate(ws) if w.nx == nx), key=lambda k: ws[k].nz)
        chs = sorted({0, ws[i].n_ch // 2, ws[i].n_ch - 1})
        picks.append((i, chs, plans[i].e0()[chs], plans[i].eh()[chs], plans[i].reflectivity()[0]))
    steps_p = max(2, steps_b // 2)
    ms_plain = timed(plain_step, steps_p, 1)
    # the plain launches recompute the same fields: alone == in the work queue
    same = all(np.array_equal(plans[i].eh()[chs], gh) and np.array_equal(plans[i].e0()[chs], g0)
               for i, chs, g0, gh, _ in picks)
    info = b.info()
    out = {
        "metric": METRIC + ", batched vs plain", "value": cells / (ms_batched * 1e-3), "unit": UNIT,
        "steps": steps_b, "warmup": 3, "ms_per_step": ms_batched,
        "workload": f"uneven batch of {len(ws)} instances (seed {3 + rank}): Nx in "
                    f"{sorted({w.nx for w in ws})}, {min(w.nz for w in ws)}-"
                    f"{max(w.nz for w in ws)} z steps, {min(w.n_ch for w in ws)}-"
                    f"{max(w.n_ch for w in ws)} channels, perfect / bent / random strain",
        "cell_updates": cells, "l2": "flushed between timed steps (256 MB write)",
        "form": "one CUDA graph: setup of every instance, persistent work-queue launches "
                "(14 queues by size and splitting order), time responses",
        "plain": {"value": cells / (ms_plain * 1e-3), "ms_per_step": ms_plain, "steps": steps_p,
                  "form": "per instance: setup kernels, one march launch in its tuned form, "
                          "time response"},
        "speedup_vs_plain": ms_plain / ms_batched,
        "plain_launch_forms": sorted({(k[0], k[1], v["form"], v["channels_per_block"])
                                      for k, v in tuned.items()}),
        "items": info["last_items"], "clocks": clocks,
        "gpu_launches": b.graph_kernels() * steps_b,
        "results_equal_batched_vs_plain": bool(same),
    }

    def parity():
        worst, rows = {}, []
        for i, chs, g0, gh, R in picks:
            e, oR = field_errors(ws[i], chs, g0, gh, jobs.threads)
            rows.append({"instance": ws[i].name, "channels": chs, **e,
                         "max_abs_err_R": float(np.max(np.abs(R[chs] - oR)))})
        for key in ("max_err_per_channel", "rel_l2_fields", "rel_l2_eh", "max_abs_err_R"):
            worst[key] = max(r[key] for r in rows)
        return {"vs": "FP64 oracle", "channels": sum(len(r["channels"]) for r in rows),
                **worst, "tolerance": TOL_FIELD, "samples": rows}

    if jobs is not None:
        jobs.submit("batched", parity)
    for p in plans:
        p.close()
    b.close()
    return out


# --------------------------------------------------------------------------- config 5
def run_3d(args, world, rank, local, jobs=None):
    """3D (x, y, z) workload: 512 x 512 transverse, 1000 steps, 128 channels,
    HBM-streamed (two passes per step, 64 B of algorithmic traffic per
    cell-update); roofline against the measured HBM copy bandwidth."""
    import torch
    from paper_2201_08500_gb300 import bpm

    torch.cuda.set_device(local)
    nz = 1000 if args.nz == 2000 else args.nz
    n_ch = 128 if args.channels == 1024 else args.channels
    w = workloads.large_3d(n_ch=n_ch, nz=nz, seed=5 + rank)
    u_host = w.u
    u_dev = torch.from_numpy(np.ascontiguousarray(u_host)).cuda()
    w.u = None
    stream = torch.cuda.current_stream()
    # launch form chosen by the autotuner (untimed setup): column-pass form and
    # row-pass tile height
    tried = []
    if args.launch_form is None:
        _, tried = bpm.tune(w.dims, w.nx, w.ny, w.dx, w.dy, w.dz, w.n_ch, steps=32)
    plan = bpm.Plan(w.dims, w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.n_ch, stream=stream)
    plan.set_timing(True)
    if args.launch_form is not None:
        plan.set_launch(form=args.launch_form, row_threads=args.row_threads)

    def step():
        plan.set_crystal(w.chi0, w.chih, w.chihb, w.theta_B, w.lambda_B, w.x_surface,
                         w.thickness, u=u_dev)
        plan.set_pulse(w.omega, w.S, w.theta_i, w.x0, w.w0, w.zx, w.zR)
        plan.run()

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    steps = max(3, min(args.steps, args.extra_steps))
    sampler = ClockSampler(local).start()
    times, march = [], []
    for i in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        plan.sync()
        times.append(e0.elapsed_time(e1))
        march.append(plan.stats()["march_ms"])
    clocks = sampler.stop()
    st = plan.stats()
    ms = statistics.median(times)
    march_ms = statistics.median(march)
    cells = w.cell_updates
    bytes_alg = 64.0 * cells
    achieved = bytes_alg / (march_ms * 1e-3) / 1e9
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    launch = plan.launch()
    out = {
        "metric": METRIC + " (omega*x*y*z), 3D", "value": cells / (ms * 1e-3), "unit": UNIT,
        "steps": steps, "warmup": 3, "ms_per_step": ms,
        "workload": w.name, "nx": w.nx, "ny": w.ny, "nz": w.nz, "channels": w.n_ch,
        "l2": "fields (512 MB) exceed L2 (129 MB)", "launch": launch, "tuned": tried,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "traffic": MEASURED_TRAFFIC_3D.get(
                         (w.name, launch["form"], launch["row_threads"])),
                     "traffic_unit": "one z step: column pass + row pass",
                     "algorithmic_bytes": 64 * w.n_ch * w.plane,
                     "kernel": {0: "row_pass_kernel + col_pass_kernel",
                                1: "row_pass_kernel + col_pass_tma_kernel",
                                2: "row_pass_tma_kernel + col_pass_tma_kernel"}[launch["form"]]
                               + " (2 passes per z step)",
                     "bytes_per_cell_update": 64, "march_ms": march_ms,
                     "passes": st["march_launches"]},
        "gpu_launches": (st["launches"] + 4) * steps, "clocks": clocks,
    }
    if jobs is not None:
        chs = [0, w.n_ch // 2]
        g0 = torch.empty((w.n_ch, w.plane), dtype=torch.complex64, device="cuda")
        gh = torch.empty_like(g0)
        plan.fetch(bpm.BPM_FIELD_E0, out=g0)
        plan.fetch(bpm.BPM_FIELD_EH, out=gh)
        g0, gh = g0[chs].cpu().numpy(), gh[chs].cpu().numpy()
        R = plan.reflectivity()[0]
        w.u = u_host

        def parity():
            e, oR = field_errors(w, chs, g0, gh, min(jobs.threads, len(chs)))
            return {"vs": "FP64 oracle", "channels": chs, **e,
                    "max_abs_err_R": float(np.max(np.abs(R[chs] - oR))),
                    "tolerance": TOL_FIELD}

        jobs.submit("3d", parity)
    plan.close()
    return out


# --------------------------------------------------------------------------- config 4
def run_served(args, world, rank, local, jobs=None):
    """Poisson stream of requests (80 % single-channel rocking-curve probes
    Nx = 512 / 300 steps, 20 % instances drawn from the uneven batch), offered at
    `load` x the measured capacity of the batched executor.  Three forms on the
    same arrivals: served with a short-request lane (4 SMs) beside the long
    lane, served with one lane, and plain (one request at a time).  Then the
    first quarter of the requests again as a burst (all arriving at once):
    served vs plain throughput at saturation."""
    import torch
    from paper_2201_08500_gb300 import bpm, serve

    torch.cuda.set_device(local)
    pool = workloads.batch(n_inst=args.instances, seed=3 + rank)
    us = [None if w.u is None else torch.from_numpy(np.ascontiguousarray(w.u)).cuda() for w in pool]
    stream = torch.cuda.current_stream()
    # capacity of the batched executor on the pool (one graph pass)
    plans = [bpm.plan_from_workload(w, stream=stream, u=u) for w, u in zip(pool, us)]
    b = bpm.Batch(stream=stream)
    for p in plans:
        b.submit(p)
    b.run_graph()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run_graph()
    torch.cuda.synchronize()
    capacity = sum(w.cell_updates for w in pool) / (time.perf_counter() - t0)
    for p in plans:
        p.close()
    b.close()
    rng = np.random.default_rng(4 + rank)
    reqs_w, reqs_u = [], []
    for i in range(args.requests):
        if rng.uniform() < 0.8:
            reqs_w.append(workloads.probe(rng, idx=i))
            reqs_u.append(None)
        else:
            j = int(rng.integers(0, len(pool)))
            reqs_w.append(pool[j])
            reqs_u.append(us[j])
    mean_cost = float(np.mean([w.cell_updates for w in reqs_w]))
    rate = args.load * capacity / mean_cost
    arr = serve.poisson_arrivals(len(reqs_w), rate, 4 + rank)

    def make(n=None, burst=False):
        n = len(reqs_w) if n is None else n
        return [serve.Request(i, w, u, 0.0 if burst else float(a))
                for i, (w, u, a) in enumerate(zip(reqs_w[:n], reqs_u[:n], arr[:n]))]

    def served_form(reqs, short_sms):
        srv = serve.Server(hbm_budget_bytes=96 * 2 ** 30, chunk=256, keep_fields=False,
                           short_sms=short_sms)
        srv.serve(reqs)
        st = serve.summarize(reqs)
        st["rounds"], st["slots"] = srv.rounds, srv.n_slots
        srv.close()
        return st

    served = make()
    sampler = ClockSampler(local).start()  # clocks during the served (headline) run
    s_stats = served_form(served, 4)
    clocks = sampler.stop()
    one = make()
    o_stats = served_form(one, 0)
    plain = make()
    p_sampler = ClockSampler(local).start()
    serve.serve_plain(plain, keep_fields=False)
    p_clocks = p_sampler.stop()
    p_stats = serve.summarize(plain)
    same = all(np.array_equal(a.R, c.R) and np.array_equal(a.R, d.R)
               for a, c, d in zip(served, plain, one))
    n_burst = max(1, len(reqs_w) // 4)
    sb = make(n_burst, burst=True)
    sb_stats = served_form(sb, 4)
    pb = make(n_burst, burst=True)
    serve.serve_plain(pb, keep_fields=False)
    pb_stats = serve.summarize(pb)
    out = {
        "metric": METRIC + " served vs plain; p50/p99 latency", "value": s_stats["throughput"],
        "unit": UNIT, "ms_per_step": s_stats["makespan_s"] * 1e3,
        "workload": f"Poisson stream of {len(served)} requests (80 % probes Nx=512 Nz=300 "
                    f"1 channel, 20 % uneven-batch instances), offered load {args.load} x "
                    f"capacity {capacity:.3e} cell-updates/s; burst: the first {n_burst} "
                    f"requests all at t = 0",
        "rate_per_s": rate, "chunk_steps": 256, "hbm_budget_gb": 96, "short_lane_sms": 4,
        "served": s_stats, "served_one_lane": o_stats, "plain": p_stats,
        "p99_ms": {"served": s_stats["p99_ms"], "served_one_lane": o_stats["p99_ms"],
                   "plain": p_stats["p99_ms"]},
        "p50_ms": {"served": s_stats["p50_ms"], "served_one_lane": o_stats["p50_ms"],
                   "plain": p_stats["p50_ms"]},
        "burst": {"served": sb_stats, "plain": pb_stats,
                  "served_vs_plain_throughput": sb_stats["throughput"] / pb_stats["throughput"]},
        "results_equal_alone_vs_mix": bool(same),
        "clocks": clocks, "clocks_plain": p_clocks,
    }
    if jobs is not None:
        probes = [r for r in served if r.work.name.startswith("probe")][:8]
        inst = []
        for r in served:
            if not r.work.name.startswith("probe") and all(r.work.name != q.work.name
                                                            for q in inst):
                inst.append(r)
            if len(inst) == 2:
                break

        def parity():
            import oracle.oracle as orc
            errs = []
            for r in probes:
                o0, oh, init = orc.run(r.work, n_threads=1)
                errs.append(float(abs(r.R[0] - orc.reflectivity(init, o0, oh)[0][0])))
            ierr = []
            for r in inst:
                chs = [0, r.work.n_ch - 1]
                o0, oh, init = orc.run(r.work, channels=chs, n_threads=min(2, jobs.threads))
                oR = orc.reflectivity(init, o0, oh)[0]
                ierr.append(float(np.max(np.abs(r.R[chs] - oR))))
            return {"vs": "FP64 oracle", "probes": len(probes),
                    "max_abs_err_R_probes": max(errs) if errs else None,
                    "instances": [r.work.name for r in inst], "channels_per_instance": 2,
                    "max_abs_err_R_instances": max(ierr) if ierr else None,
                    "note": "R_i of requests served in the mix (first served form)"}

        jobs.submit("served", parity)
    return out


# --------------------------------------------------------------------------- config 2
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="N = 1: skip the nested batched / served / 3d objects")
    ap.add_argument("--extra-steps", type=int, default=5,
                    help="timed passes of the batched and 3d sections (at most --steps)")
    ap.add_argument("--channels", type=int, default=1024,
                    help="channels of the deformed workload (profiling: a smaller instance)")
    ap.add_argument("--nz", type=int, default=2000, help="z steps of the deformed workload")
    ap.add_argument("--nx", type=int, default=4096, help="transform size of the deformed workload")
    ap.add_argument("--row-threads", type=int, default=None, choices=[128, 256, 512],
                    help="with --launch-form on the 3d workload: the row-pass tile")
    ap.add_argument("--launch-form", type=int, default=None, choices=[0, 1, 2, 3],
                    help="force a launch form of the deformed workload's march (default: "
                         "the autotuner's choice)")
    ap.add_argument("--split-order", type=int, default=1, choices=[1, 2, 4],
                    help="operator splitting of the deformed workload (Eq. split-op)")
    ap.add_argument("--workload", default="deformed", choices=["deformed", "batched", "served", "3d"],
                    help="deformed: one instance (default line); batched / served / 3d: that "
                         "section alone, as its own line")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--requests", type=int, default=10000,
                    help="served: number of requests (80 % rocking-curve probes)")
    ap.add_argument("--load", type=float, default=0.7, help="served: offered load / capacity")
    ap.add_argument("--independent", action="store_true",
                    help="N > 1: every rank marches its own instance (weak scaling) instead of "
                         "the ranks splitting one instance's channels")
    ap.add_argument("--shard-channels", action="store_true",
                    help="split one instance's channels across the ranks (the default at N > 1)")
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    single = {"batched": run_batched, "served": run_served, "3d": run_3d}
    if args.workload in single:
        obj = single[args.workload](args, world, rank, local)
        if rank == 0:
            print(json.dumps({"n_gpus": world, "data": "synthetic", **obj}), flush=True)
        return 0

    import torch
    from paper_2201_08500_gb300 import bpm, shard

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    peaks = measure_cuda_core_peaks(local)
    sharded = world > 1 and not args.independent
    w_all = None  # the sharded instance
    if sharded:
        w, w_all, first = rank_share(args.channels, args.nx, args.nz, world, rank)
    else:
        w = rank_workload(args.channels, args.nx, args.nz, rank)
    w.split_order = args.split_order
    stream = torch.cuda.current_stream()
    u_dev = torch.from_numpy(np.ascontiguousarray(w.u)).cuda()
    # launch form chosen by the autotuner (untimed setup); 256 steps: short runs
    # over-weight the one-time per-channel table copy of the shared-memory form
    tried = []
    if args.launch_form is None:
        _, tried = bpm.tune(w.dims, w.nx, w.ny, w.dx, w.dy, w.dz, w.n_ch,
                            split_order=w.split_order, steps=min(w.nz, 256))
    plan = bpm.Plan(w.dims, w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.n_ch, stream=stream,
                    zassenhaus=w.zassenhaus, split_order=w.split_order)
    plan.set_timing(True)
    if sharded:
        plan.set_channel_shard(first, w_all.n_ch, shard.pulse_spacing(w_all.omega))
        t_dev = torch.empty((w_all.n_ch, w.plane), dtype=torch.complex128, device="cuda")
    if args.launch_form is not None:
        # the parked forms run one channel per block; the TMEM form at
        # Nx = 1024 two
        cpb = (2 if args.launch_form == 3 and w.nx == 1024 else 1) if args.launch_form >= 2 else None
        plan.set_launch(form=args.launch_form, channels_per_block=cpb)
    omega = np.ascontiguousarray(w.omega)
    S = np.ascontiguousarray(w.S)
    rows = {}

    def step(u):
        plan.set_crystal(w.chi0, w.chih, w.chihb, w.theta_B, w.lambda_B, w.x_surface,
                         w.thickness, u=u)
        plan.set_pulse(omega, S, w.theta_i, w.x0, w.w0, w.zx, w.zR)
        plan.run()
        if sharded:
            # the one exchange of a sharded pulse: reduce-scatter the time
            # response over t (each rank keeps its block of time rows)
            plan.fetch(bpm.BPM_FIELD_EH_TIME, out=t_dev)
            rows["t"], rows["first"], _ = shard.combine_scatter(t_dev, 0.0)

    # L2 (129 MB) is flushed between timed steps by writing a 256 MB buffer
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    for _ in range(max(3, args.warmup)):
        step(u_dev)
    barrier()

    sampler = ClockSampler(local).start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    march_ms = []
    barrier()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step(u_dev)
        ev[i][1].record(stream)
        plan.sync()
        march_ms.append(plan.stats()["march_ms"])
    barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms_local = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms_local, dist, device="cuda")
    cells_per_rank = w.cell_updates
    # whole-job cell-updates: every rank's instance, or the one sharded instance
    job_cells = w_all.cell_updates if sharded else world * cells_per_rank
    value = whole_job_value(1, job_cells, ms)

    # end to end through the C ABI with host buffers: pinned u in, R and the
    # time response (this rank's rows of it when sharded) out, copies inside
    # the timed region
    u_pin = torch.from_numpy(np.ascontiguousarray(w.u)).pin_memory()
    t_rows = w.n_ch
    if sharded:
        t_rows = rows["t"].shape[0]
    t_host = torch.empty((t_rows, w.plane), dtype=torch.complex128).pin_memory()
    R = np.empty(w.n_ch)
    e2e_ms = []
    for i in range(max(2, min(args.steps, 5))):
        barrier()
        t0 = time.perf_counter()
        step(u_pin)
        if sharded:
            t_host.copy_(rows["t"])
        else:
            plan.fetch(bpm.BPM_FIELD_EH_TIME, out=t_host)
        R, _, _ = plan.reflectivity()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = max_over_ranks(statistics.median(e2e_ms), dist, device="cuda")
    h2d = w.u.nbytes + omega.nbytes + S.nbytes
    d2h = t_host.numel() * t_host.element_size() + 2 * R.nbytes

    st = plan.stats()
    n = w.nx
    march_avg = statistics.mean(march_ms)
    achieved = cells_per_rank * flops_per_cell(n, w.split_order) / (march_avg * 1e-3) / 1e12
    # algorithmic DRAM bytes of one launch: tables (32 B per channel and x), fields
    # in and out (32 B), one read of the deformation rows (8 B per x and step)
    sets = 2 if w.split_order == 4 else 1
    alg_bytes = w.n_ch * n * (32 * sets + 32) + w.nz * n * 8
    form = plan.launch()["form"]
    kernel = f"march_kernel<{n},{st['channels_per_block']}> form {form}"
    props = torch.cuda.get_device_properties(local)
    pk = measured_peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    peak_units = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    peak = peaks["fp32"]["tflops"]
    executed = EXECUTED_FLOPS.get(kernel) if w.split_order == 1 else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong" if sharded else "weak",
            "vs_baseline": None,
            "dtype": "c64 fields / f32 butterflies (f64 setup and time sum)",
            "data": "synthetic",
            "config": {"workload": w_all.name if sharded else w.name, "nx": w.nx, "nz": w.nz,
                       "channels": w_all.n_ch if sharded else w.n_ch,
                       "split_order": w.split_order,
                       "crystal": "thermal bump u = A exp(-x'^2/w^2)(z/Z)^2",
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": (f"{world} x channel shard of one instance, time "
                                       f"response reduce-scattered over t" if sharded
                                       else f"{world} x independent instance"),
                       "launch": plan.launch(), "tuned": tried},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "peak_basis": "measured FP32 FFMA rate on every SM (peaks.fp32, "
                                       "bpm_measure_peak)",
                         "peak_unit_count": peak_units,
                         "frac_unit_count": achieved / peak_units,
                         "unit_count_basis": f"{props.multi_processor_count} SMs x 128 FP32 "
                                             f"lanes x 2 x {sm_max:.0f} MHz",
                         "flops_per_cell_update": flops_per_cell(n, w.split_order),
                         "flops_basis": "nominal: 4 FFTs at 5 N log2 N + 12 + 40 per cell-update",
                         "executed_flops_per_cell_update": executed,
                         "frac_executed": (None if executed is None else
                                           cells_per_rank * executed / (march_avg * 1e-3)
                                           / 1e12 / peak),
                         "executed_basis": "ncu FADD + FMUL + 2 FFMA thread instructions of "
                                           "this kernel per cell-update",
                         # the captured launch held the whole instance
                         "traffic": (MEASURED_TRAFFIC.get((kernel, w.name, w.split_order))
                                     if not sharded else None),
                         "algorithmic_bytes": alg_bytes,
                         "kernel": kernel, "march_ms": march_avg},
            "peaks": peaks,
            "e2e": {"value": job_cells / (e2e * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": 5 * args.steps,
            "clocks": clocks,
        }
        if not args.no_cpu_baseline and world == 1:
            cores = os.cpu_count() or 1
            # about 10 s of CPU work: 12 channels per core, full march
            n_s = max(1, min(w.n_ch, 12 * cores))
            v, dt, cells, (idx, o0, oh, init) = oracle_sample(w, n_s, cores, keep=True)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": f"{n_s} of {w.n_ch} channels spread over the band, "
                                              f"full {w.nz}-step march ({dt:.1f} s)"}
            # error of the GPU's FP32 fields (the last bench step, z = Nz) on the same
            # channels, per channel relative to the incident field's norm
            g0, gh = plan.e0()[idx], plan.eh()[idx]
            line["parity"] = {"vs": "FP64 oracle", "channels": int(n_s),
                              **parity_figures(g0, gh, o0, oh, init), "tolerance": TOL_FIELD}
    plan.close()
    del u_dev, flush
    if world == 1 and not args.no_extras:
        # each section is reported on its own: one that fails records its
        # error in the line instead of costing the others (or the main line)
        torch.cuda.empty_cache()
        jobs = OracleJobs(threads=max(1, (os.cpu_count() or 2) - 4))
        extras = {}
        t_x = time.perf_counter()
        for name, fn in (("batched", run_batched), ("3d", run_3d), ("served", run_served)):
            try:
                extras[name] = fn(args, world, rank, local, jobs)
            except Exception as e:  # noqa: BLE001 - reported in the line
                extras[name] = {"error": repr(e)[:400]}
            try:
                torch.cuda.synchronize()
                torch.cuda.empty_cache()
            except Exception as e:  # noqa: BLE001 - a lost context ends the sections
                extras[name].setdefault("error", repr(e)[:400])
                break
        for name in extras:
            if "error" not in extras[name] and name in jobs.jobs:
                extras[name]["parity"] = jobs.result(name)
        jobs.close()
        line.update(extras)
        line["extras_wall_s"] = time.perf_counter() - t_x
        line["gpu_launches_extras"] = {k: extras[k].get("gpu_launches") for k in extras}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
