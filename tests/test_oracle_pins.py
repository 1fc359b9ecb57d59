"""Pins for the CPU oracle: things the paper and the mathematics fix, not the
oracle's own formulas retyped.

  * brute force: per-nanosecond tick counting on tiny traces equals the
    oracle's unions and host sums exactly;
  * closed forms: balanced devices give LB = 1, one device / one rank give
    LB = 1, disjoint kernels and transfers hide nothing, transfers inside
    kernels cost nothing, a covering kernel is the kernel time, union <= sum,
    a tiled host gives E = window length and CE_host = 1 iff the most loaded
    rank has no MPI time;
  * invariants: every ratio in [0, 1] on tiled inputs and each parent equal
    to the product of its children (Eqs. 3-5 and 6-12 multiply out);
  * the paper's synthetic-benchmark tables (Sec. 5.1, PILS use cases 1-7):
    two-rank traces rebuilt from each use case's narrative reproduce every
    printed value to the printed two decimals;
  * the printed tables of Sec. 5.1 and 5.2 themselves satisfy the
    parent = product-of-children identities within their rounding;
  * the host tree with threads (a variant the paper does not define): one
    thread per process gives the paper's host tree bit for bit, a worked
    example by hand, processes of identical threads, per-ns ticks for its
    integer aggregates, bounds, identities and permutation invariance.

Every pin is a function of an oracle build, so test_oracle_mutants.py can run
the same pins against deliberately broken builds and check that each one is
caught.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import tracegen as tg
from fractions import Fraction

from helpers import (GOLDEN, fixture_trace, host_tiles_windows, host_units_trace, load_fixture, pils_cases,
                     tick_device, tick_host, tick_concurrency)

pytestmark = pytest.mark.filterwarnings("ignore")

RATIOS = oracle.RATIO_FIELDS


# ----------------------------------------------------------------------------
# pins as functions of an oracle instance


def pin_brute_force(O, seeds=range(60)):
    for seed in seeds:
        t = tg.tiny_trace(seed)
        for r in range(t.n_regions):
            du = O.device_unions(t, r)
            np.testing.assert_array_equal(du, tick_device(t, r), err_msg=f"device unions seed={seed} r={r}")
            hs = O.host_sums(t, r)
            np.testing.assert_array_equal(hs, tick_host(t, r), err_msg=f"host sums seed={seed} r={r}")


def _balanced_trace(seed):
    t = tg.tiny_trace(seed, max_ranks=3, max_devs=2, allow_empty=False, tiled_host=True)
    # give every device the records of device 0 and every rank the same window
    se0, tag0 = t.dev_segment(0)
    m = t.m_devices
    dev_se = np.concatenate([se0] * m)
    dev_tag = np.concatenate([tag0] * m)
    dev_off = np.arange(m + 1, dtype=np.uint64) * np.uint64(se0.shape[0])
    win = t.region_window.copy()
    win[:, :, :] = win[:, :1, :]
    return tg.Trace(trace_id=0, n_ranks=t.n_ranks, devices_per_rank=t.devices_per_rank, region_window=win,
                    host_se=t.host_se, host_state=t.host_state, host_off=t.host_off,
                    dev_se=dev_se, dev_tag=dev_tag, dev_off=dev_off)


def pin_balanced_devices_lb_one(O):
    for seed in range(20):
        t = _balanced_trace(seed)
        for r in range(t.n_regions):
            res = O.region_metrics(t, r)
            if res["max_kernel"] > 0:
                assert res["dev_lb"] == 1.0, (seed, r, res["dev_lb"])


def pin_single_unit_lb_one(O):
    for seed in range(40):
        t = tg.tiny_trace(seed, max_ranks=1, max_devs=1, allow_empty=False)
        for r in range(t.n_regions):
            res = O.region_metrics(t, r)
            assert res["dev_lb"] == 1.0 and res["host_mpi_lb"] == 1.0, (seed, r, res)


def _kernel_transfer_trace(inside: bool, seed=0):
    """One rank, one device: kernels on a grid; transfers either strictly in
    the gaps (disjoint) or strictly inside kernels."""
    rng = np.random.default_rng(seed)
    ks = np.arange(0, 100) * 1000
    kd = rng.integers(100, 600, 100)
    recs = [(int(s), int(s + d), 0, 0) for s, d in zip(ks, kd)]
    mems = []
    for s, d in zip(ks, kd):
        if inside:
            a = int(s + rng.integers(0, d // 2))
            b = int(a + rng.integers(0, d - (a - s)))
        else:
            a = int(s + d + rng.integers(0, 100))
            b = int(a + rng.integers(0, 1000 - d - (a - s - d)))
        mems.append((a, b, 1 + int(rng.integers(0, 4)), 1))
    recs = sorted(recs + mems)
    T = 100_000
    fx = dict(n_ranks=1, devices_per_rank=[1], window=[[0, T]], host=[[[0, T, 0]]],
              device=[[list(r) for r in recs]])
    return fixture_trace(fx), sum(b - a for a, b, _, _ in mems)


def pin_disjoint_transfers_not_hidden(O):
    for seed in range(5):
        t, msum = _kernel_transfer_trace(inside=False, seed=seed)
        res = O.region_metrics(t, 0)
        assert res["sum_hidden_mem"] == 0
        assert res["sum_mem"] == msum


def pin_transfers_inside_kernels_cost_nothing(O):
    for seed in range(5):
        t, _ = _kernel_transfer_trace(inside=True, seed=seed)
        res = O.region_metrics(t, 0)
        assert res["sum_mem"] == 0
        assert res["dev_ce"] == 1.0


def pin_covering_kernel(O):
    for seed in range(20):
        t = tg.tiny_trace(seed, max_ranks=1, max_devs=1, allow_empty=False, kinds=(0,))
        se, tag = t.dev_segment(0)
        lo, hi = int(se[:, 0].min()), int(se[:, 1].max()) + 7
        big = np.array([[lo, hi]], np.int64)
        t2 = tg.Trace(trace_id=0, n_ranks=1, devices_per_rank=t.devices_per_rank,
                      region_window=np.array([[[-10**9, 10**9]]], np.int64),
                      host_se=t.host_se, host_state=t.host_state, host_off=t.host_off,
                      dev_se=np.concatenate([big, se]), dev_tag=np.concatenate([np.zeros(1, np.uint8), tag]),
                      dev_off=np.array([0, se.shape[0] + 1], np.uint64))
        du = O.device_unions(t2, 0)
        assert du[0, 0] == hi - lo and du[0, 2] == hi - lo, (seed, du)


def pin_union_at_most_sum(O):
    for seed in range(40):
        t = tg.tiny_trace(seed)
        for r in range(t.n_regions):
            du = O.device_unions(t, r)
            win = t.region_window[r]
            g = 0
            for i in range(t.n_ranks):
                a, b = win[i]
                for _ in range(int(t.devices_per_rank[i])):
                    se, tag = t.dev_segment(g)
                    clip = np.clip(np.minimum(se[:, 1], b) - np.maximum(se[:, 0], a), 0, None)
                    kind = tag >> 5
                    assert du[g, 0] <= clip[kind == 0].sum()
                    assert du[g, 1] <= clip[kind != 0].sum()
                    assert max(du[g, 0], du[g, 1]) <= du[g, 2] <= du[g, 0] + du[g, 1]
                    assert du[g, 2] <= max(b - a, 0)
                    g += 1


def pin_tiled_host_elapsed_and_ce(O):
    for seed in range(40):
        t = tg.tiny_trace(seed, tiled_host=True, allow_empty=False)
        if not host_tiles_windows(t, 0):
            continue
        res = O.region_metrics(t, 0)
        win = t.region_window[0]
        assert res["elapsed_ns"] == int((win[:, 1] - win[:, 0]).max())
        hs = O.host_sums(t, 0)
        uw = hs[:, 0] + hs[:, 1]
        top = np.flatnonzero(uw == uw.max())
        full = win[:, 1] - win[:, 0]
        ce_one = any(hs[i, 2] == 0 and full[i] == res["elapsed_ns"] for i in top)
        assert (res["host_mpi_ce"] == 1.0) == ce_one, (seed, res, hs)
        assert res["flags"] & oracle.FLAG_HOST_NOT_TILED == 0


def _check_invariants(res, tag):
    for k in RATIOS:
        assert 0.0 <= res[k] <= 1.0, (tag, k, res[k])
    eps = 4 * np.finfo(np.float64).eps
    pairs = [(res["host_pe"], res["host_mpi_pe"] * res["host_oe"]),
             (res["host_mpi_pe"], res["host_mpi_lb"] * res["host_mpi_ce"]),
             (res["dev_pe"], res["dev_lb"] * res["dev_ce"] * res["dev_oe"])]
    for a, b in pairs:
        assert abs(a - b) <= eps * max(abs(a), abs(b)) + 1e-300, (tag, a, b, res)


def pin_invariants(O):
    for seed in range(40):
        t = tg.tiny_trace(seed, tiled_host=True)
        if host_tiles_windows(t, 0):
            _check_invariants(O.region_metrics(t, 0), ("tiny", seed))
    for seed in range(3):
        t = tg.random_trace(seed, dev_events=400, host_events=300, n_regions=4)
        for r in range(t.n_regions):
            _check_invariants(O.region_metrics(t, r), ("random", seed, r))


def pin_pils_tables(O):
    for path in pils_cases():
        fx = load_fixture(path)
        res = O.region_metrics(fixture_trace(fx), 0)
        for k, v in fx["printed"].items():
            assert abs(res[k] - v) <= 0.005 + 1e-12, (fx["name"], k, res[k], v)


def pin_empty_and_degenerate(O):
    # no records at all: E = 0, every ratio 1, EMPTY flag
    fx = dict(n_ranks=2, devices_per_rank=[1, 0], window=[[0, 0], [5, 5]], host=[[], []], device=[[]])
    res = O.region_metrics(fixture_trace(fx), 0)
    assert res["elapsed_ns"] == 0 and res["flags"] & oracle.FLAG_EMPTY
    assert all(res[k] == 1.0 for k in RATIOS)
    # host only, no devices: device ratios reported as 1 with NO_DEVICES
    fx = dict(n_ranks=1, devices_per_rank=[0], window=[[0, 10]], host=[[[0, 4, 0], [4, 10, 2]]], device=[])
    res = O.region_metrics(fixture_trace(fx), 0)
    assert res["flags"] & oracle.FLAG_NO_DEVICES and res["dev_pe"] == 1.0
    assert res["host_pe"] == 0.4 and res["host_mpi_ce"] == 0.4
    # devices with only transfers: D_K = 0 -> PE_dev = 0, LB_dev = 1 (0/0), CE_dev = 0
    fx = dict(n_ranks=1, devices_per_rank=[1], window=[[0, 10]], host=[[[0, 10, 1]]],
              device=[[[2, 6, 1, 0]]])
    res = O.region_metrics(fixture_trace(fx), 0)
    assert (res["dev_pe"], res["dev_lb"], res["dev_ce"], res["dev_oe"]) == (0.0, 1.0, 0.0, 0.4)
    assert res["host_pe"] == 0.0 and res["host_oe"] == 0.0 and res["sum_idle"] == 6


def pin_validation(O):
    t = tg.tiny_trace(5, allow_empty=False)
    assert O.validate(t) == 0
    bad = tg.Trace(**{**t.__dict__})
    bad.dev_se = t.dev_se.copy()
    bad.dev_se[0] = (10, 9)
    assert O.validate(bad) & 4
    bad.dev_se = t.dev_se
    bad.dev_tag = t.dev_tag.copy()
    bad.dev_tag[0] = 5 << 5
    assert O.validate(bad) & 8


def pin_concurrency_brute_force(O, seeds=range(40)):
    """Concurrency profile = per-ns counts of active records, on tiny traces."""
    for seed in seeds:
        t = tg.tiny_trace(seed, trace_id=seed, max_events=80, horizon=600)
        for r in range(t.n_regions):
            np.testing.assert_array_equal(O.concurrency(t, r, 6), tick_concurrency(t, r, 6), err_msg=str((seed, r)))


def pin_concurrency_closed_forms(O):
    """Level 1 is the busy (kernel) union; the levels add up to the summed
    record time; k identical records give k levels of their length; nested
    records give level 2 = the inner one; back-to-back records never reach 2."""
    for seed in range(10):
        t = tg.random_trace(seed, trace_id=seed, n_ranks=2, devices_per_rank=2, dev_events=700, host_events=50,
                            n_regions=3)
        for r in range(t.n_regions):
            c = O.concurrency(t, r, 64)
            u = O.device_unions(t, r)
            np.testing.assert_array_equal(c[:, 0, 0], u[:, 2])
            np.testing.assert_array_equal(c[:, 1, 0], u[:, 0])
            win = t.region_window[r]
            dr = np.repeat(np.arange(t.n_ranks), t.devices_per_rank)
            for g in range(t.m_devices):
                a, b = int(t.dev_off[g]), int(t.dev_off[g + 1])
                lo, hi = win[dr[g], 0], win[dr[g], 1]
                se = t.dev_se[a:b]
                ln = np.maximum(np.minimum(se[:, 1], hi) - np.maximum(se[:, 0], lo), 0)
                assert c[g, 0].sum() == ln.sum() and c[g, 0, -1] == 0
                assert c[g, 1].sum() == ln[(t.dev_tag[a:b] >> 5) == 0].sum()
    base = dict(trace_id=1, n_ranks=1, devices_per_rank=np.array([1], np.uint32),
                region_window=np.array([[[0, 1000]]], np.int64), host_se=np.zeros((0, 2), np.int64),
                host_state=np.zeros(0, np.uint8), host_off=np.array([0, 0], np.uint64))
    same = tg.Trace(dev_se=np.array([[100, 400]] * 5, np.int64), dev_tag=np.array([0, 0, 0, 32, 64], np.uint8),
                    dev_off=np.array([0, 5], np.uint64), **base)
    c = O.concurrency(same, 0, 8)
    assert c[0, 0].tolist() == [300] * 5 + [0] * 3 and c[0, 1].tolist() == [300] * 3 + [0] * 5
    nest = tg.Trace(dev_se=np.array([[100, 900], [200, 300], [250, 260]], np.int64),
                    dev_tag=np.array([0, 0, 0], np.uint8), dev_off=np.array([0, 3], np.uint64), **base)
    assert O.concurrency(nest, 0, 4)[0, 0].tolist() == [800, 100, 10, 0]
    chain = tg.Trace(dev_se=np.array([[0, 100], [100, 250], [250, 251], [300, 2000]], np.int64),
                     dev_tag=np.array([0, 32, 0, 64], np.uint8), dev_off=np.array([0, 4], np.uint64), **base)
    assert O.concurrency(chain, 0, 3)[0, 0].tolist() == [951, 0, 0]      # clipped at 1000


def _runs(O, ns=(1, 2, 4, 8), gpus=(1, 2, 2, 3)):
    return [O.region_metrics(tg.random_trace(40 + k, trace_id=k, n_ranks=n, devices_per_rank=g, dev_events=400,
                                             host_events=300, n_regions=2), 1) for k, (n, g) in enumerate(zip(ns, gpus))]


def pin_scalability_identities(O):
    """Reference run: speedup and scalabilities 1, global = parallel
    efficiency.  Strong scaling: GE_r = PE_ref * speedup_r * n_ref / n_r
    (m for the device); weak scaling: GE_r = PE_ref * speedup_r."""
    runs = _runs(O)
    for ref in (0, 2):
        for weak in (False, True):
            sc = O.scalability(runs, ref, weak)
            assert sc[ref]["speedup"] == 1.0 and sc[ref]["host_comp_scal"] == 1.0 and sc[ref]["dev_comp_scal"] == 1.0
            assert sc[ref]["host_global_eff"] == runs[ref]["host_pe"]
            assert sc[ref]["dev_global_eff"] == runs[ref]["dev_pe"]
            for r, x in enumerate(sc):
                fh = 1.0 if weak else runs[ref]["n_ranks"] / runs[r]["n_ranks"]
                fd = 1.0 if weak else runs[ref]["m_devices"] / runs[r]["m_devices"]
                assert math.isclose(x["host_global_eff"], runs[ref]["host_pe"] * x["speedup"] * fh, rel_tol=1e-13)
                assert math.isclose(x["dev_global_eff"], runs[ref]["dev_pe"] * x["speedup"] * fd, rel_tol=1e-13)
                assert math.isclose(x["speedup"], runs[ref]["elapsed_ns"] / runs[r]["elapsed_ns"], rel_tol=1e-15)


def pin_scalability_closed_forms(O):
    """A run that repeats the reference on twice the ranks (same elapsed
    time, twice the useful and kernel time): strong scalability 1/2, weak
    scalability 1, speedup 1."""
    t = tg.random_trace(77, trace_id=1, n_ranks=2, devices_per_rank=[1, 3], dev_events=[300, 200, 500, 100],
                        host_events=[200, 250], n_regions=1)
    def twice(a, off):
        return np.concatenate([a, a]), np.concatenate([off[:-1], off[:-1] + off[-1], [2 * off[-1]]]).astype(np.uint64)
    hse, hoff = twice(t.host_se, t.host_off)
    dse, doff = twice(t.dev_se, t.dev_off)
    t2 = tg.Trace(trace_id=2, n_ranks=4, devices_per_rank=np.tile(t.devices_per_rank, 2),
                  region_window=np.concatenate([t.region_window, t.region_window], axis=1), host_se=hse,
                  host_state=np.concatenate([t.host_state, t.host_state]), host_off=hoff, dev_se=dse,
                  dev_tag=np.concatenate([t.dev_tag, t.dev_tag]), dev_off=doff)
    runs = [O.region_metrics(t, 0), O.region_metrics(t2, 0)]
    strong = O.scalability(runs, 0, False)[1]
    weak = O.scalability(runs, 0, True)[1]
    assert strong["speedup"] == 1.0 and strong["host_comp_scal"] == 0.5 and strong["dev_comp_scal"] == 0.5
    assert weak["speedup"] == 1.0 and weak["host_comp_scal"] == 1.0 and weak["dev_comp_scal"] == 1.0
    assert weak["host_global_eff"] == runs[1]["host_pe"] == runs[0]["host_pe"]


# ----------------------------------------------------------------------------
# host tree with threads

THREAD_TREE = (("pe", "host_pe"), ("mpi_pe", "host_mpi_pe"), ("mpi_lb", "host_mpi_lb"),
               ("mpi_ce", "host_mpi_ce"), ("oe", "host_oe"))


def pin_threads_one_per_process(O):
    """One thread per process is the paper's host tree, bit for bit."""
    for seed in range(40):
        t = tg.tiny_trace(seed)
        po = np.arange(t.n_ranks + 1, dtype=np.uint32)
        for r in range(t.n_regions):
            a, b = O.region_metrics(t, r), O.thread_metrics(t, r, po)
            assert (b["elapsed_ns"], b["sum_useful"], b["sum_offload"]) == \
                (a["elapsed_ns"], a["sum_useful"], a["sum_offload"]), (seed, r)
            assert b["max_busiest"] == a["max_useful_offload"] and b["n_threads"] == a["n_ranks"]
            for x, y in THREAD_TREE:
                assert b[x] == a[y], (seed, r, x, b[x], a[y])
            assert b["thread_lb"] == 1.0


def pin_threads_worked_example(O):
    """Two processes on [0, 100): process 0 = threads {U 40, W 20, MPI 35} and
    {U 50, W 20, MPI 28}; process 1 = {U 30, MPI 60}, {U 20}, {U 10, MPI 20}.
    By hand: E = 98 (the second thread of process 0: 50 + 20 + 28); busiest
    threads M = 70 (a worker, not the master's 60) and 30; sum_i T_i M_i =
    2*70 + 3*30 = 230; sum U = 150, sum W = 40, nT = 5.  So PE = 150/490,
    MPI PE = 230/490, MPI LB = 230/350, MPI CE = 70/98, thread LB = 190/230,
    OE = 150/190 (every denominator exact, so each value is the correctly
    rounded fraction)."""
    fx = dict(n_ranks=5, devices_per_rank=[0] * 5, window=[[0, 100]] * 5,
              host=[[[0, 40, 0], [40, 60, 1], [60, 95, 2]], [[0, 50, 0], [50, 70, 1], [70, 98, 2]],
                    [[0, 30, 0], [30, 90, 2]], [[0, 20, 0]], [[0, 10, 0], [10, 30, 2]]], device=[])
    res = O.thread_metrics(fixture_trace(fx), 0, [0, 2, 5])
    got = tuple(res[k] for k in ("elapsed_ns", "sum_useful", "sum_offload", "sum_busiest", "max_busiest", "n_threads"))
    assert got == (98, 150, 40, 230, 70, 5), got
    want = dict(pe=Fraction(150, 490), mpi_pe=Fraction(230, 490), mpi_lb=Fraction(230, 350),
                mpi_ce=Fraction(70, 98), thread_lb=Fraction(190, 230), oe=Fraction(150, 190))
    for k, v in want.items():
        assert res[k] == float(v), (k, res[k], float(v))
    assert res["flags"] == 0


def pin_threads_replicated(O):
    """A process of T identical threads: thread LB = 1, and the rest equal the
    paper's tree of the one-thread trace (every sum and nT scale by T)."""
    for seed in range(20):
        t = tg.tiny_trace(seed, allow_empty=False)
        T = [1 + (seed + i) % 4 for i in range(t.n_ranks)]
        if len(set(T)) > 1 and seed % 2:
            T = [T[0]] * t.n_ranks          # uniform T: every factor carries over
        order = [i for i in range(t.n_ranks) for _ in range(T[i])]
        rep = host_units_trace(t, order)
        po = np.zeros(t.n_ranks + 1, np.uint32)
        po[1:] = np.cumsum(T)
        base = host_units_trace(t, range(t.n_ranks))
        for r in range(t.n_regions):
            a, b = O.region_metrics(base, r), O.thread_metrics(rep, r, po)
            assert b["thread_lb"] == 1.0 and b["elapsed_ns"] == a["elapsed_ns"]
            assert b["sum_busiest"] == sum(Ti * m for Ti, m in zip(T, (O.host_sums(base, r)[:, :2].sum(1))))
            if len(set(T)) == 1:
                for x, y in THREAD_TREE:
                    assert math.isclose(b[x], a[y], rel_tol=4e-16, abs_tol=1e-300), (seed, r, x, b[x], a[y])


def _random_groups(rng, n):
    cuts = np.sort(rng.choice(np.arange(1, n), size=int(rng.integers(0, n)), replace=False)) if n > 1 else []
    return np.concatenate([[0], cuts, [n]]).astype(np.uint32)


def pin_threads_brute_force(O):
    """Integer aggregates of the thread tree from per-ns ticks, with the host
    units of tiny traces cut into processes at random."""
    for seed in range(30):
        t = tg.tiny_trace(seed, max_ranks=6)
        po = _random_groups(np.random.default_rng(seed), t.n_ranks)
        for r in range(t.n_regions):
            ticks = tick_host(t, r)
            busy = ticks[:, 0] + ticks[:, 1]
            M = [int(busy[a:b].max()) for a, b in zip(po[:-1], po[1:])]
            T = np.diff(po.astype(np.int64))
            res = O.thread_metrics(t, r, po)
            assert res["elapsed_ns"] == int(ticks.sum(1).max(initial=0)), (seed, r)
            assert res["sum_busiest"] == int(sum(Ti * m for Ti, m in zip(T, M))), (seed, r)
            assert res["max_busiest"] == max(M) and res["n_threads"] == t.n_ranks and res["n_procs"] == len(M)
            assert res["sum_useful"] == ticks[:, 0].sum() and res["sum_offload"] == ticks[:, 1].sum()


def pin_threads_invariants(O):
    """Every factor in [0, 1]; PE = MPI PE x thread LB x OE and MPI PE = MPI LB
    x MPI CE within rounding; permuting the processes, or the threads inside
    a process, changes no value."""
    eps = 4 * np.finfo(np.float64).eps
    for seed in range(6):
        rng = np.random.default_rng(100 + seed)
        base = tg.random_trace(seed, trace_id=seed, n_ranks=3, devices_per_rank=1, dev_events=50, host_events=200,
                               n_regions=3)
        t = tg.add_threads(base, [1 + seed % 3, 3, 5], seed=seed)
        po = t.meta["proc_off"]
        procs = [list(range(a, b)) for a, b in zip(po[:-1], po[1:])]
        perm = [procs[i] for i in rng.permutation(len(procs))]
        perm = [list(rng.permutation(p)) for p in perm]
        pt = host_units_trace(t, [u for p in perm for u in p])
        ppo = np.concatenate([[0], np.cumsum([len(p) for p in perm])]).astype(np.uint32)
        for r in range(t.n_regions):
            res = O.thread_metrics(t, r, po)
            for k in oracle.THREAD_RATIO_FIELDS:
                assert 0.0 <= res[k] <= 1.0, (seed, r, k, res[k])
            for a, b in ((res["pe"], res["mpi_pe"] * res["thread_lb"] * res["oe"]),
                         (res["mpi_pe"], res["mpi_lb"] * res["mpi_ce"])):
                assert abs(a - b) <= eps * max(abs(a), abs(b)), (seed, r, a, b)
            assert O.thread_metrics(pt, r, ppo) == res, (seed, r)
            assert res["thread_lb"] < 1.0      # workers are idle part of the time


def pin_threads_empty(O):
    """No host time: E = 0, EMPTY, every ratio 1; a process whose threads are
    all idle has M = 0 and counts towards nT only."""
    fx = dict(n_ranks=3, devices_per_rank=[0] * 3, window=[[0, 10]] * 3, host=[[], [], []], device=[])
    res = O.thread_metrics(fixture_trace(fx), 0, [0, 1, 3])
    assert res["elapsed_ns"] == 0 and res["flags"] == 1 and all(res[k] == 1.0 for k in oracle.THREAD_RATIO_FIELDS)
    fx["host"] = [[[0, 10, 0]], [], []]
    res = O.thread_metrics(fixture_trace(fx), 0, [0, 1, 3])
    assert (res["pe"], res["mpi_pe"], res["mpi_lb"], res["mpi_ce"], res["thread_lb"], res["oe"]) == \
        (10 / 30, 10 / 30, 10 / 30, 1.0, 1.0, 1.0)


ALL_PINS = [pin_brute_force, pin_balanced_devices_lb_one, pin_single_unit_lb_one,
            pin_disjoint_transfers_not_hidden, pin_transfers_inside_kernels_cost_nothing, pin_covering_kernel,
            pin_union_at_most_sum, pin_tiled_host_elapsed_and_ce, pin_invariants, pin_pils_tables,
            pin_empty_and_degenerate, pin_validation, pin_concurrency_brute_force, pin_concurrency_closed_forms,
            pin_scalability_identities, pin_scalability_closed_forms, pin_threads_one_per_process,
            pin_threads_worked_example, pin_threads_replicated, pin_threads_brute_force, pin_threads_invariants,
            pin_threads_empty]


# ----------------------------------------------------------------------------
# the tests (default oracle build)


def test_concurrency_brute_force_many_seeds():
    pin_concurrency_brute_force(oracle.default(), seeds=range(40, 200))


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin):
    pin(oracle.default())


def _interval(v):
    return (v - 0.005, v + 0.005)


def _mul(*ivs):
    lo = math.prod(a for a, _ in ivs)
    hi = math.prod(b for _, b in ivs)
    return lo, hi


def test_printed_tables_multiply_out():
    """Sec. 5.1/5.2 tables: PE_host = MPI_PE x OE_host, MPI_PE = LB x CE (LB
    and CE take offloading as useful), PE_dev = LB x CE x OE_dev, each within
    the two-decimal rounding of the printed values."""
    data = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))
    assert len(data["columns"]) == 20
    for c in data["columns"]:
        for parent, kids in [("host_pe", ("host_mpi_pe", "host_oe")),
                             ("host_mpi_pe", ("host_mpi_lb", "host_mpi_ce")),
                             ("dev_pe", ("dev_lb", "dev_ce", "dev_oe"))]:
            lo, hi = _mul(*[_interval(c[k]) for k in kids])
            plo, phi = _interval(c[parent])
            assert lo <= phi + 1e-12 and plo <= hi + 1e-12, (c["source"], parent, c[parent], lo, hi)


def test_brute_force_many_seeds():
    pin_brute_force(oracle.default(), seeds=range(60, 400))
