"""GPU path vs the CPU oracle, element by element (bit-exact), through the C ABI.

Sizes span several tiles per warp and ragged tails; the sweep shapes and the
number of tiles per warp are varied so that slices start inside device
segments (exercising the fix-up of the carry) and segments are shorter than
a tile.
"""
import numpy as np
import pytest

import oracle
import tracegen as tg
from gpu_common import assert_metrics_equal, assert_trace_equal, make_ctx
from helpers import fixture_trace, load_fixture, pils_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    c.close()


def test_tiny_traces_one_by_one(ctx):
    for seed in range(60):
        t = tg.tiny_trace(seed, trace_id=seed)
        ctx.ingest([t])
        assert_trace_equal(ctx, t, "tiny")
    ctx.reset()


def test_tiny_traces_batched_many_warps():
    c = make_ctx(tiles_per_warp=1)
    try:
        ts = [tg.tiny_trace(seed, trace_id=seed) for seed in range(400)]
        c.ingest(ts)
        for t in ts:
            assert_trace_equal(c, t, "tiny-batched", sums=(t.trace_id % 7 == 0))
    finally:
        c.close()


def test_pils_fixtures(ctx):
    for k, path in enumerate(pils_cases()):
        fx = load_fixture(path)
        t = fixture_trace(fx, trace_id=1000 + k)
        ctx.ingest([t])
        res = ctx.metrics(t.trace_id)[0]
        assert_metrics_equal(res, oracle.region_metrics(t, 0), fx["name"])
        for key, v in fx["printed"].items():
            assert abs(res[key] - v) <= 0.005 + 1e-12, (fx["name"], key, res[key], v)
    ctx.reset()


def test_single_trace_small_full_size(ctx):
    t = tg.single_trace_small()
    ctx.ingest([t], flags=2)  # caller asserts start order
    assert_trace_equal(ctx, t, "4x1x1 10k")
    ctx.reset()


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
@pytest.mark.parametrize("tpw", [1, 3, 64])
def test_random_traces_shapes(shape, tpw):
    c = make_ctx(shape=shape, tiles_per_warp=tpw)
    try:
        for seed in range(3):
            t = tg.random_trace(seed + 10 * shape, trace_id=seed, n_ranks=3, devices_per_rank=[1, 2, 3],
                                dev_events=[2000 + 37 * seed, 5000, 1, 0, 333, 7000], host_events=[4000, 1, 2500],
                                n_regions=3 + seed)
            c.ingest([t])
            assert_trace_equal(c, t, ("shape", shape, tpw, seed))
    finally:
        c.close()


@pytest.mark.parametrize("spw", [1, 5, 64])
def test_slices_handed_out_by_ticket(spw):
    """The sweep's dynamic work split (slices of the records taken by warps
    as they come free, a record per slice for the fix-up): mid-size traces,
    long covering intervals and records out of start order (the first
    sweep's run log and the sort stage) equal the oracle under 1, 5 and 64
    slices per warp and one tile per warp."""
    c = make_ctx(tiles_per_warp=1, slices_per_warp=spw)
    try:
        for seed in range(2):
            t = tg.random_trace(seed + 70, trace_id=seed, n_ranks=3, devices_per_rank=[1, 2, 3],
                                dev_events=[2000 + 37 * seed, 5000, 1, 0, 333, 7000], host_events=[4000, 1, 2500],
                                n_regions=5)
            c.ingest([t])
            assert_trace_equal(c, t, ("slices", spw, seed))
            c.ingest([_covering_trace(seed + 20)])
            assert_trace_equal(c, _covering_trace(seed + 20), ("slices covering", spw, seed))
            u = tg.split_runs(tg.random_trace(seed + 80, trace_id=40 + seed, n_ranks=2, devices_per_rank=2,
                                              dev_events=9000, host_events=300, n_regions=3), 4, seed=seed)
            c.ingest([u])
            assert_trace_equal(c, u, ("slices unsorted", spw, seed))
            c.reset()
    finally:
        c.close()


def _covering_trace(seed, n=20000):
    """Long kernels and copies that span many tiles and warps: the carry
    entering a slice can reach far ahead."""
    rng = np.random.default_rng(seed)
    s = np.sort(rng.integers(0, 10_000_000, n))
    d = rng.integers(0, 2000, n)
    big = rng.random(n) < 0.002
    d[big] = rng.integers(100_000, 5_000_000, big.sum())
    kind = np.where(rng.random(n) < 0.6, 0, rng.integers(1, 5, n)).astype(np.uint8)
    se = np.stack([s, s + d], 1).astype(np.int64)
    tag = tg.make_tag(kind, rng.integers(0, 8, n))
    T = int(se[:, 1].max()) + 1
    host = np.array([[0, T // 3], [T // 3, T]], np.int64)
    win = np.array([[[0, T]], [[T // 5, T // 2]], [[T // 2, T // 2 + 1000]]], np.int64)
    return tg.Trace(trace_id=seed, n_ranks=1, devices_per_rank=np.array([1], np.uint32), region_window=win,
                    host_se=host, host_state=np.array([0, 1], np.uint8), host_off=np.array([0, 2], np.uint64),
                    dev_se=se, dev_tag=tag, dev_off=np.array([0, n], np.uint64))


@pytest.mark.parametrize("tpw", [1, 2, 1000])
def test_covering_intervals_cross_slices(tpw):
    c = make_ctx(tiles_per_warp=tpw)
    try:
        for seed in range(4):
            t = _covering_trace(seed)
            c.ingest([t])
            assert_trace_equal(c, t, ("covering", tpw, seed))
    finally:
        c.close()


@pytest.mark.parametrize("scale,offset", [(1 << 20, 0), (1 << 28, 0), (3, (1 << 61) + 12345),
                                          (1 << 21, -(1 << 58))])
def test_wide_timestamps_take_the_exact_path(scale, offset):
    """Spans of 2^32 ns and more (the int64 path of the sweep), values near
    2^61 and negative times; mixed with tiles that fit 32-bit offsets."""
    c = make_ctx(tiles_per_warp=1)
    try:
        ts = [tg.rescale_time(tg.tiny_trace(seed, trace_id=seed, max_events=300), scale, offset)
              for seed in range(40)]
        c.ingest(ts)
        for t in ts:
            assert_trace_equal(c, t, ("wide", scale, offset), sums=(t.trace_id % 5 == 0))
        for seed in range(2):
            t = tg.rescale_time(_covering_trace(seed, n=6000), scale, offset)
            c.ingest([t])
            assert_trace_equal(c, t, ("wide-covering", scale, offset, seed))
    finally:
        c.close()


def test_device_pointers_match_host_pointers(ctx):
    import torch
    t = tg.random_trace(5, trace_id=77, n_ranks=4, devices_per_rank=2, dev_events=3000, host_events=2000,
                        n_regions=4)
    arrays = [dict(host_se=torch.from_numpy(t.host_se).cuda(), host_state=torch.from_numpy(t.host_state).cuda(),
                   dev_se=torch.from_numpy(t.dev_se).cuda(), dev_tag=torch.from_numpy(t.dev_tag).cuda())]
    ctx.ingest([t], arrays=arrays)
    torch.cuda.synchronize()
    assert_trace_equal(ctx, t, "device-ptrs")
    ctx.reset()


def _split_by_time(t, frac):
    """Two time slices of a trace: records starting before the cut, the rest."""
    cut = int(np.quantile(t.dev_se[:, 0], frac)) if t.n_dev else 0
    parts = []
    for first in (True, False):
        dse, dtg, doff = [], [], [0]
        for g in range(t.m_devices):
            se, tag = t.dev_segment(g)
            sel = se[:, 0] < cut if first else se[:, 0] >= cut
            dse.append(se[sel])
            dtg.append(tag[sel])
            doff.append(doff[-1] + int(sel.sum()))
        hse, hst, hoff = [], [], [0]
        for i in range(t.n_ranks):
            se, st = t.host_segment(i)
            sel = se[:, 0] < cut if first else se[:, 0] >= cut
            hse.append(se[sel])
            hst.append(st[sel])
            hoff.append(hoff[-1] + int(sel.sum()))
        parts.append(tg.Trace(trace_id=t.trace_id, n_ranks=t.n_ranks, devices_per_rank=t.devices_per_rank,
                              region_window=t.region_window, host_se=np.concatenate(hse),
                              host_state=np.concatenate(hst), host_off=np.asarray(hoff, np.uint64),
                              dev_se=np.concatenate(dse), dev_tag=np.concatenate(dtg),
                              dev_off=np.asarray(doff, np.uint64)))
    return parts


@pytest.mark.parametrize("tpw", [1, 8])
def test_append_slices_equal_whole(tpw):
    c = make_ctx(tiles_per_warp=tpw)
    try:
        t = tg.random_trace(9, trace_id=5, n_ranks=3, devices_per_rank=2, dev_events=6000, host_events=3000,
                            n_regions=4)
        a, b = _split_by_time(t, 0.4)
        c.ingest([a])
        c.ingest([b], flags=4)  # APPEND
        assert_trace_equal(c, t, ("append", tpw))
        # out-of-order append (an earlier slice after a later one) is reported
        c.ingest([b])
        c.ingest([a], flags=4)
        st, _ = c.metrics(5, check=False)
        assert st == -1
    finally:
        c.close()


def test_invalid_records_are_reported(ctx):
    t = tg.random_trace(3, trace_id=11, n_ranks=2, devices_per_rank=1, dev_events=500, host_events=300)
    bad = tg.Trace(**{**t.__dict__})
    bad.dev_se = t.dev_se.copy()
    bad.dev_se[17] = (bad.dev_se[17, 0], bad.dev_se[17, 0] - 1)
    ctx.ingest([bad])
    st, res = ctx.metrics(11, check=False)
    assert st == -1 and res[0]["flags"] & 0x100
    bad.dev_se = t.dev_se
    bad.dev_tag = t.dev_tag.copy()
    bad.dev_tag[3] = 6 << 5
    ctx.ingest([bad])
    st, res = ctx.metrics(11, check=False)
    assert st == -1 and res[0]["flags"] & 0x100
    bad.dev_tag = t.dev_tag
    bad.host_state = t.host_state.copy()
    bad.host_state[5] = 3
    ctx.ingest([bad])
    st, res = ctx.metrics(11, check=False)
    assert st == -1 and res[0]["flags"] & 0x100
    # a valid ingest of the same id replaces the state and the status
    ctx.ingest([t])
    assert_trace_equal(ctx, t, "after-invalid")
    ctx.reset()


def test_sorted_flag_with_unsorted_records_is_reported(ctx):
    t = tg.shuffle_segments(tg.random_trace(4, trace_id=12, n_ranks=2, devices_per_rank=2, dev_events=800,
                                            host_events=100), seed=3)
    ctx.ingest([t], flags=2)
    st, res = ctx.metrics(12, check=False)
    assert st == -1 and res[0]["flags"] & 0x200
    ctx.reset()


def test_header_errors_are_immediate(ctx):
    import paper_2603_26576_b300 as P
    t = tg.tiny_trace(1, trace_id=13)
    b, keep = P.batch_from_arrays(13, t.devices_per_rank, t.region_window, t.host_se, t.host_state, t.host_off,
                                  t.dev_se, t.dev_tag, t.dev_off)
    b.n_regions = 9
    with pytest.raises(P.TalpGpuError) as ei:
        P.talp_gpu_ingest_events(ctx.ctx, [b])
    assert ei.value.status == -1
    with pytest.raises(P.TalpGpuError) as ei:
        P.talp_gpu_region_metrics(ctx.ctx, 987654, 0)
    assert ei.value.status == -5


def test_admission_refuses_over_budget():
    import paper_2603_26576_b300 as P
    c = make_ctx(budget=4 << 20)
    try:
        t = tg.random_trace(1, trace_id=1, n_ranks=2, devices_per_rank=1, dev_events=300_000, host_events=10)
        with pytest.raises(P.TalpGpuError) as ei:
            c.ingest([t])
        assert ei.value.status == -2
        held, budget = c.memory()
        assert held <= budget
        small = tg.tiny_trace(2, trace_id=2)
        c.ingest([small])
        assert_trace_equal(c, small, "after-admission")
    finally:
        c.close()


def test_metrics_batch_and_reset(ctx):
    ts = [tg.tiny_trace(s, trace_id=100 + s, n_regions=2) for s in range(5)]
    ctx.ingest(ts)
    res = ctx.metrics_batch([t.trace_id for t in ts], 1)
    for t, r in zip(ts, res):
        assert_metrics_equal(r, oracle.region_metrics(t, 1), ("batch", t.trace_id))
    held0, _ = ctx.memory()
    ctx.reset(100)
    held1, _ = ctx.memory()
    assert held1 < held0
    ctx.reset()
