"""Host-side arithmetic of bench.py (no GPU): the nominal flop counts the
rooflines divide by, the parity figures against the oracle, the whole-job
value and the channel shares of a sharded pulse."""
import math
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_nominal_flops_count_propagations_and_couplings():
    # order 1: one propagation (4 FFTs of 5 N log2 N over N cells, two table
    # products) and one coupling (40); Strang adds a coupling; fourth order
    # has three propagations and four couplings (Eq. split-op)
    for n in (256, 1024, 4096, 8192):
        fft = 4 * 5 * n * math.log2(n) / n
        prop = fft + 2 * 6
        assert bench.flops_per_cell(n, 1) == pytest.approx(prop + 40)
        assert bench.flops_per_cell(n, 2) == pytest.approx(prop + 2 * 40)
        assert bench.flops_per_cell(n, 4) == pytest.approx(3 * prop + 4 * 40)
    assert bench.flops_per_cell(4096) == 292.0


def test_parity_figures_of_a_known_perturbation():
    rng = np.random.default_rng(7)
    n_ch, n = 5, 64
    o0 = rng.normal(size=(n_ch, n)) + 1j * rng.normal(size=(n_ch, n))
    oh = rng.normal(size=(n_ch, n)) + 1j * rng.normal(size=(n_ch, n))
    init = 2.0 * (rng.normal(size=(n_ch, n)) + 1j * rng.normal(size=(n_ch, n)))
    exact = bench.parity_figures(o0, oh, o0, oh, init)
    assert exact["max_err_per_channel"] == 0.0 and exact["rel_l2_fields"] == 0.0
    # one cell of channel 3's Eh off by d: per-channel error d / |init_3|,
    # the other channels exact (median 0), rel-L2 figures d / |field|
    d = 1e-3
    gh = oh.copy()
    gh[3, 10] += d
    f = bench.parity_figures(o0, gh, o0, oh, init)
    assert f["max_err_per_channel"] == pytest.approx(d / np.linalg.norm(init[3]))
    assert f["median_err_per_channel"] == 0.0
    assert f["rel_l2_eh"] == pytest.approx(d / np.linalg.norm(oh))
    both = math.sqrt(np.linalg.norm(o0) ** 2 + np.linalg.norm(oh) ** 2)
    assert f["rel_l2_fields"] == pytest.approx(d / both)
    # an E0 error of the same size in the same channel does not add to the
    # per-channel figure (the larger of the two envelopes' errors)
    g0 = o0.copy()
    g0[3, 20] -= d
    f2 = bench.parity_figures(g0, gh, o0, oh, init)
    assert f2["max_err_per_channel"] == pytest.approx(f["max_err_per_channel"])
    # the figures are relative: scaling everything leaves them unchanged
    s = 1e5
    f3 = bench.parity_figures(s * g0, s * gh, s * o0, s * oh, s * init)
    for k in ("max_err_per_channel", "rel_l2_fields", "rel_l2_eh"):
        assert f3[k] == pytest.approx(f2[k])


def test_whole_job_value_divides_every_rank_by_the_slowest_time():
    assert bench.whole_job_value(1, 10**9, 1000.0) == pytest.approx(1e9)
    assert bench.whole_job_value(4, 10**9, 500.0) == pytest.approx(8e9)
    assert bench.max_over_ranks(3.5) == 3.5  # no process group: identity


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_rank_shares_cover_the_pulse_once(world):
    n_ch, nx, nz = 13, 256, 4
    seen = []
    for rank in range(world):
        w, w_all, first = bench.rank_share(n_ch, nx, nz, world, rank)
        assert w_all.n_ch == n_ch and w.nx == nx and w.nz == nz
        assert np.array_equal(w.omega, w_all.omega[first:first + w.n_ch])
        seen.extend(range(first, first + w.n_ch))
    assert seen == list(range(n_ch))
