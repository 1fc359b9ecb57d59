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
    parent = product-of-children identities within their rounding.

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
from helpers import (GOLDEN, fixture_trace, host_tiles_windows, load_fixture, pils_cases, tick_device,
                     tick_host, tick_concurrency)

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


ALL_PINS = [pin_brute_force, pin_balanced_devices_lb_one, pin_single_unit_lb_one,
            pin_disjoint_transfers_not_hidden, pin_transfers_inside_kernels_cost_nothing, pin_covering_kernel,
            pin_union_at_most_sum, pin_tiled_host_elapsed_and_ce, pin_invariants, pin_pils_tables,
            pin_empty_and_degenerate, pin_validation, pin_concurrency_brute_force, pin_concurrency_closed_forms,
            pin_scalability_identities, pin_scalability_closed_forms]


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
