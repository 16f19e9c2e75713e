"""GPU tests of the batched (work-queue) and continuous-batching forms.

Each plan in a batch runs the same per-channel code as a single-plan launch, so
its fields must equal the single-plan result bitwise (alone vs in the mix), and
the oracle within the parity tolerance on sampled channels."""
import numpy as np
import pytest

import oracle.oracle as orc
from paper_2201_08500_gb300 import bpm, workloads

pytestmark = pytest.mark.gpu

TOL_FIELD = 1e-4


@pytest.fixture(scope="module")
def stream():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    return torch.cuda.current_stream()


def mix(seed=21):
    """Six uneven instances: every batch transform size, perfect / bent / random strain."""
    rng = np.random.default_rng(seed)
    spec = [(1024, 130, 12, "bent"), (2048, 90, 7, "random"), (4096, 60, 5, "perfect"),
            (8192, 40, 3, "random"), (512, 150, 20, "bent"), (256, 170, 33, "random")]
    out = []
    for i, (nx, nz, nch, kind) in enumerate(spec):
        w = workloads.mixed_instance(rng, nx=nx, nz=nz, n_ch=nch, kind=kind, idx=i)
        # bring the beam near the surface so that both envelopes carry power
        w.x0 = w.x_surface - 30 * w.dx
        w.w0 = 10 * w.dx
        out.append(w)
    return out


def single(w, stream):
    p = bpm.plan_from_workload(w, stream=stream)
    p.run()
    p.sync()
    r = dict(e0=p.e0(), eh=p.eh(), R=p.reflectivity()[0], t=p.eh_time())
    p.close()
    return r


def fetch(p):
    return dict(e0=p.e0(), eh=p.eh(), R=p.reflectivity()[0], t=p.eh_time())


def assert_same(a, b):
    for k in ("e0", "eh", "R", "t"):
        assert np.array_equal(a[k], b[k]), k


def test_batch_alone_vs_mix_and_oracle(stream):
    ws = mix()
    ref = [single(w, stream) for w in ws]
    b = bpm.Batch(stream=stream)
    plans = [bpm.plan_from_workload(w, stream=stream) for w in ws]
    tickets = [b.submit(p) for p in plans]
    b.run()
    b.sync()
    info = b.info()
    assert info["rounds"] == 1 and info["last_items"][1] > 0  # the Nx = 8192 queue ran
    for t, p, r in zip(tickets, plans, ref):
        assert b.poll(t)
        assert_same(fetch(p), r)
    for w, r in zip(ws, ref):
        pick = [0, w.n_ch - 1]
        o0, oh, init = orc.run(w.subset(pick))
        inc = np.linalg.norm(init, axis=1)
        err = max(np.max(np.linalg.norm(r["e0"][pick] - o0, axis=1) / inc),
                  np.max(np.linalg.norm(r["eh"][pick] - oh, axis=1) / inc))
        assert err < TOL_FIELD, (w.name, err)
        assert np.linalg.norm(oh) > 1e-3 * np.linalg.norm(init)
    for p in plans:
        p.close()
    b.close()


def test_chunked_rounds_equal_one_round(stream):
    ws = mix(seed=5)[:4]
    ref = [single(w, stream) for w in ws]
    b = bpm.Batch(stream=stream)
    plans = [bpm.plan_from_workload(w, stream=stream) for w in ws]
    tickets = [b.submit(p) for p in plans]
    done = [False] * len(plans)
    rounds = 0
    while not all(done):
        b.step(23)
        rounds += 1
        b.sync()
        done = [b.poll(t) if not d else True for t, d in zip(tickets, done)]
        assert rounds < 100
    assert rounds == -(-max(w.nz for w in ws) // 23)
    for p, r in zip(plans, ref):
        assert_same(fetch(p), r)
        p.close()
    b.close()


def test_continuous_admission_joins_later_rounds(stream):
    """A plan submitted while others are mid-march joins the next round and gives
    the same result as alone; admission is bounded by the byte budget."""
    ws = mix(seed=8)
    ref = [single(w, stream) for w in ws[:3]]
    sizes = [bpm.plan_bytes(w.dims, w.nx, w.ny, w.nz, w.n_ch, host_u=w.u is not None)
             for w in ws[:3]]
    b = bpm.Batch(hbm_budget_bytes=sizes[0] + sizes[1] + sizes[2] // 2, stream=stream)
    p0 = bpm.plan_from_workload(ws[0], stream=stream)
    p1 = bpm.plan_from_workload(ws[1], stream=stream)
    p2 = bpm.plan_from_workload(ws[2], stream=stream)
    t0 = b.submit(p0)
    b.step(40)
    t1 = b.submit(p1)  # joins mid-way
    assert b.try_submit(p2) is None  # budget full: not admitted
    t2 = None
    for _ in range(200):
        b.step(40)
        b.sync()
        if t2 is None and b.poll(t0):
            t2 = b.submit(p2)  # admitted once p0's share was released
        if t2 is not None and b.poll(t1) and b.poll(t2):
            break
    assert t2 is not None
    for p, r in zip((p0, p1, p2), ref):
        assert_same(fetch(p), r)
        p.close()
    b.close()


def test_cancel_releases_budget(stream):
    ws = mix(seed=2)[:2]
    b = bpm.Batch(stream=stream)
    p0 = bpm.plan_from_workload(ws[0], stream=stream)
    p1 = bpm.plan_from_workload(ws[1], stream=stream)
    t0, t1 = b.submit(p0), b.submit(p1)
    used = b.info()["used_bytes"]
    b.step(10)
    b.cancel(t0)
    assert b.info()["used_bytes"] < used
    with pytest.raises(bpm.BpmError):
        b.poll(t0)
    b.run()
    b.sync()
    assert b.poll(t1)
    assert_same(fetch(p1), single(ws[1], stream))
    p0.close()
    p1.close()
    b.close()


def test_graph_replay_equals_eager(stream):
    import torch
    ws = mix(seed=13)
    ref = [single(w, stream) for w in ws]
    us = [None if w.u is None else torch.from_numpy(np.ascontiguousarray(w.u)).cuda() for w in ws]
    plans = [bpm.plan_from_workload(w, stream=stream, u=u) for w, u in zip(ws, us)]
    b = bpm.Batch(stream=stream)
    for p in plans:
        b.submit(p)
    assert b.graph_kernels() == 0
    for _ in range(3):  # capture, then replay twice
        b.run_graph()
        b.sync()
        for p, r in zip(plans, ref):
            assert_same(fetch(p), r)
    # per plan at least tables, incident field and time response; two march queues
    assert b.graph_kernels() >= 3 * len(plans) + 2
    for p in plans:
        p.close()
    b.close()


def test_strang_plans_in_a_mixed_batch(stream):
    ws = mix(seed=17)[:3]
    ws[1].split_order = 2
    ref = [single(w, stream) for w in ws]
    b = bpm.Batch(stream=stream)
    plans = [bpm.plan_from_workload(w, stream=stream) for w in ws]
    for p in plans:
        b.submit(p)
    b.run()
    b.sync()
    for p, r in zip(plans, ref):
        assert_same(fetch(p), r)
        p.close()
    b.close()


def test_fourth_order_plans_in_a_mixed_batch(stream):
    """Fourth-order plans (Eq. split-op, t = 1/(2 - 2^(1/3))) at Nx = 1024, 8192
    and 256 share the batch with first- and second-order plans: each equals its
    single-plan march bitwise, and the oracle on sampled channels."""
    ws = mix(seed=23)
    for i in (0, 3, 5):
        ws[i].split_order = 4
    ws[1].split_order = 2
    ref = [single(w, stream) for w in ws]
    b = bpm.Batch(stream=stream)
    plans = [bpm.plan_from_workload(w, stream=stream) for w in ws]
    for p in plans:
        b.submit(p)
    b.run()
    b.sync()
    for p, r in zip(plans, ref):
        assert_same(fetch(p), r)
        p.close()
    b.close()
    for i in (0, 3):
        w, r = ws[i], ref[i]
        pick = [0, w.n_ch - 1]
        o0, oh, init = orc.run(w.subset(pick))
        inc = np.linalg.norm(init, axis=1)
        err = max(np.max(np.linalg.norm(r["e0"][pick] - o0, axis=1) / inc),
                  np.max(np.linalg.norm(r["eh"][pick] - oh, axis=1) / inc))
        assert err < TOL_FIELD, (w.name, err)


def test_strang_and_fourth_order_parked_queues(stream):
    """The parked queues of the higher orders: Strang at Nx = 2048, 4096, 8192
    (tables in TMEM) and fourth order at Nx = 1024, 2048, 4096 (tables from
    L2), in one batch; each plan equals its single-plan march bitwise."""
    ws = mix(seed=31)[:4] + mix(seed=37)[:3]   # Nx 1024, 2048, 4096, 8192, 1024, 2048, 4096
    for w, order in zip(ws, (4, 2, 2, 2, 4, 4, 4)):
        w.split_order = order
    ref = [single(w, stream) for w in ws]
    b = bpm.Batch(stream=stream)
    plans = [bpm.plan_from_workload(w, stream=stream) for w in ws]
    for p in plans:
        b.submit(p)
    b.run()
    b.sync()
    for p, r in zip(plans, ref):
        assert_same(fetch(p), r)
        p.close()
    b.close()


def test_block_cap_and_rounds_in_flight(stream):
    """A batch capped at 3 blocks gives the same fields; pending() counts rounds
    whose kernels have not finished and is 0 after a sync."""
    ws = mix(seed=8)[:3]
    ref = [single(w, stream) for w in ws]
    b = bpm.Batch(stream=stream)
    b.set_max_blocks(3)
    plans = [bpm.plan_from_workload(w, stream=stream) for w in ws]
    tickets = [b.submit(p) for p in plans]
    assert b.pending() == 0
    for _ in range(3):
        b.step(50)
    assert 0 <= b.pending() <= 3
    b.run()
    b.sync()
    assert b.pending() == 0
    for t, p, r in zip(tickets, plans, ref):
        assert b.poll(t)
        assert_same(fetch(p), r)
        p.close()
    b.close()


def test_full_uneven_batch_sampled_against_oracle(stream):
    """The uneven batch at its full size (64 instances, seed 3, Nx 1024..8192,
    Nz 500..4000, 128..1024 channels: the workload the batched bench times, in
    one graph-captured pass): sampled channels of the largest transform and of
    the longest march, plus a mid-size instance, against the oracle."""
    import torch
    ws = workloads.batch(n_inst=64, seed=3)
    us = [None if w.u is None else torch.from_numpy(np.ascontiguousarray(w.u)).cuda()
          for w in ws]
    b = bpm.Batch(stream=stream)
    plans = [bpm.plan_from_workload(w, stream=stream, u=u) for w, u in zip(ws, us)]
    for p in plans:
        b.submit(p)
    b.run_graph()
    b.sync()
    big = max(range(len(ws)), key=lambda i: (ws[i].nx, ws[i].nz))
    longest = max(range(len(ws)), key=lambda i: ws[i].nz * ws[i].nx)
    mid = next(i for i, w in enumerate(ws) if w.nx == 2048)
    for i in sorted({big, longest, mid}):
        w = ws[i]
        pick = [w.n_ch // 2, w.n_ch - 1]
        o0, oh, init = orc.run(w.subset(pick))
        g0, gh = plans[i].e0()[pick], plans[i].eh()[pick]
        inc = np.linalg.norm(init, axis=1)
        err = max(np.max(np.linalg.norm(g0 - o0, axis=1) / inc),
                  np.max(np.linalg.norm(gh - oh, axis=1) / inc))
        assert err < TOL_FIELD, (i, w.nx, w.nz, err)
    for p in plans:
        p.close()
    b.close()
