"""The sort stage: device records out of start order (no SORTED_BY_START
flag) are sorted on the GPU and the results equal the oracle bit for bit."""
import numpy as np
import pytest

import oracle
import tracegen as tg
from gpu_common import assert_metrics_equal, assert_trace_equal, make_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    c.close()


def test_shuffled_tiny_traces_batched(ctx):
    ts = [tg.shuffle_segments(tg.tiny_trace(seed, trace_id=seed, max_events=200), seed=seed, frac=0.7)
          for seed in range(120)]
    ctx.ingest(ts)
    for t in ts:
        assert_trace_equal(ctx, t, "shuffled-tiny", sums=(t.trace_id % 4 == 0))
    ctx.reset()


@pytest.mark.parametrize("mode", ["lanes", "shuffle"])
def test_unsorted_mid_size(ctx, mode):
    for seed in range(3):
        base = tg.random_trace(seed, trace_id=seed, n_ranks=3, devices_per_rank=[2, 1, 3],
                               dev_events=[9000, 1, 0, 20000, 5000, 4097], host_events=[3000, 10, 7], n_regions=4)
        t = tg.interleave_lanes(base) if mode == "lanes" else tg.shuffle_segments(base, seed=seed)
        ctx.ingest([t])
        assert_trace_equal(ctx, t, (mode, seed))
    ctx.reset()


@pytest.mark.parametrize("k", [2, 3, 5, 16, 17, 40])
def test_few_sorted_runs(ctx, k):
    """Segments made of k sorted runs: up to 16 runs take the merge path,
    more the radix path; ties across runs, one-record runs and segments
    shorter and longer than a sort tile included."""
    for seed in range(2):
        base = tg.random_trace(seed + 10 * k, trace_id=seed, n_ranks=3, devices_per_rank=[2, 1, 3],
                               dev_events=[9000, 2, 1, 20000, 5000, 4097], host_events=[300, 10, 7], n_regions=3)
        t = tg.split_runs(base, k, seed=seed)
        ctx.ingest([t])
        assert_trace_equal(ctx, t, ("runs", k, seed))
    ts = [tg.split_runs(tg.tiny_trace(s, trace_id=s, max_events=300, horizon=512), k, seed=s) for s in range(40)]
    ctx.ingest(ts)
    for t in ts:
        assert_trace_equal(ctx, t, ("runs-tiny", k), sums=(t.trace_id % 3 == 0))
    ctx.reset()


def test_unsorted_wide_timestamps(ctx):
    """Keys spanning many radix digits (up to 8 passes)."""
    for scale, offset in [(1 << 30, 0), (1 << 45, -(1 << 61)), (7, (1 << 61))]:
        ts = [tg.shuffle_segments(tg.rescale_time(tg.tiny_trace(s, trace_id=s, max_events=300), scale, offset), seed=s)
              for s in range(20)]
        ctx.ingest(ts)
        for t in ts:
            assert_trace_equal(ctx, t, ("wide-unsorted", scale), sums=(t.trace_id % 5 == 0))
    ctx.reset()


@pytest.mark.parametrize("k", [2, 4, 7, 16])
def test_few_sorted_runs_wide_timestamps(ctx, k):
    """k-run segments whose starts span 2^50 to 2^57 ns or sit near -2^61:
    the merge path compares full 64-bit starts in its splits and merges."""
    for scale, offset in [(1 << 45, -(1 << 61)), (1 << 40, 0), (1 << 38, 5)]:
        ts = [tg.split_runs(tg.rescale_time(tg.tiny_trace(s, trace_id=s, max_events=400), scale, offset), k, seed=s)
              for s in range(16)]
        ctx.ingest(ts)
        for t in ts:
            assert_trace_equal(ctx, t, ("wide-runs", k, scale), sums=(t.trace_id % 4 == 0))
        ctx.reset()


def test_mixed_sorted_and_unsorted_batches(ctx):
    """One ingest call with traces that assert start order and traces that
    do not; a trace that asserts order but lies is still reported."""
    good = [tg.tiny_trace(s, trace_id=100 + s) for s in range(10)]
    uns = [tg.shuffle_segments(tg.tiny_trace(s, trace_id=200 + s), seed=s) for s in range(10)]
    import paper_2603_26576_b300 as P
    batches, keep = [], []
    for t in good:
        b, k = P.batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, t.host_se, t.host_state,
                                   t.host_off, t.dev_se, t.dev_tag, t.dev_off, P.TALP_GPU_SORTED_BY_START)
        batches.append(b)
        keep.append(k)
    for t in uns:
        b, k = P.batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, t.host_se, t.host_state,
                                   t.host_off, t.dev_se, t.dev_tag, t.dev_off, 0)
        batches.append(b)
        keep.append(k)
    liar = tg.shuffle_segments(tg.tiny_trace(3, trace_id=300, allow_empty=False, max_events=60), seed=9)
    b, k = P.batch_from_arrays(liar.trace_id, liar.devices_per_rank, liar.region_window, liar.host_se,
                               liar.host_state, liar.host_off, liar.dev_se, liar.dev_tag, liar.dev_off,
                               P.TALP_GPU_SORTED_BY_START)
    batches.append(b)
    keep.append(k)
    P.talp_gpu_ingest_events(ctx.ctx, batches)
    for t in good + uns:
        ctx._shapes[int(t.trace_id)] = (t.n_ranks, t.m_devices, t.n_regions)
        assert_trace_equal(ctx, t, "mixed", sums=False)
    ctx._shapes[300] = (liar.n_ranks, liar.m_devices, liar.n_regions)
    st, res = ctx.metrics(300, check=False)
    unsorted_somewhere = any(np.any(np.diff(liar.dev_segment(g)[0][:, 0]) < 0) for g in range(liar.m_devices))
    if unsorted_somewhere:
        assert st == -1 and res[0]["flags"] & 0x200
    ctx.reset()


def test_append_with_unsorted_slices():
    """Each later slice arrives out of order inside itself (sorted on the GPU);
    the earlier slices' sums are kept."""
    from test_gpu_parity import _split_by_time
    c = make_ctx(tiles_per_warp=1)
    try:
        t = tg.random_trace(12, trace_id=7, n_ranks=2, devices_per_rank=2, dev_events=5000, host_events=2000,
                            n_regions=3)
        a, b = _split_by_time(t, 0.5)
        c.ingest([tg.interleave_lanes(a)])
        c.ingest([tg.shuffle_segments(b, seed=4)], flags=4)
        assert_trace_equal(c, t, "append-unsorted")
        # a slice that starts before the previous one ended is still refused
        c.ingest([tg.interleave_lanes(b)])
        c.ingest([tg.shuffle_segments(a, seed=5)], flags=4)
        st, _ = c.metrics(7, check=False)
        assert st == -1
    finally:
        c.close()


def test_unsorted_with_many_warps_per_segment():
    c = make_ctx(tiles_per_warp=1)
    try:
        base = tg.random_trace(31, trace_id=1, n_ranks=1, devices_per_rank=1, dev_events=300_000,
                               host_events=1000, n_regions=2)
        t = tg.interleave_lanes(base)
        c.ingest([t])
        assert_trace_equal(c, t, "unsorted-big")
    finally:
        c.close()


def _runs_of_sizes(trace, sizes, seed):
    """The trace's one device segment dealt into sorted runs of the given
    sizes (records drawn at random for each run, each run in start order),
    laid end to end: the start order descends only where a run begins."""
    rng = np.random.default_rng(seed)
    n = int(trace.dev_off[1])
    assert sum(sizes) == n
    grp = rng.permutation(np.repeat(np.arange(len(sizes)), sizes))
    order = np.argsort(grp, kind="stable")
    se, tag = trace.dev_se.copy(), trace.dev_tag.copy()
    se[:n], tag[:n] = se[:n][order], tag[:n][order]
    return tg._with_dev(trace, se, tag)


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
def test_run_boundaries_at_tile_and_slice_edges(shape):
    """The first sweep logs where each device's start order descends (inside
    a tile, at a tile's first record, at a warp slice's first record through
    the fix-up, in tiles it only scans after the segment is found out of
    order); with one tile per warp every tile edge is a slice edge.  Runs
    that begin exactly there, one-record runs, and 15 / 16 / 17 descents
    (16 runs is the most the fused merge-sweep takes) all equal the oracle."""
    tile = 32 * (9, 7, 11, 13)[shape]     # records per tile of each sweep shape
    c = make_ctx(shape=shape, tiles_per_warp=1)
    try:
        for k in (2, 15, 16, 17):
            for variant in range(3):
                if variant == 0:     # every run a whole number of tiles
                    sizes = [tile * (1 + (i % 3)) for i in range(k)]
                elif variant == 1:   # runs one record off a tile edge, and one-record runs
                    sizes = [tile + (1 if i % 2 else -1) if i % 4 else 1 for i in range(k)]
                else:                # runs of random lengths
                    sizes = list(np.random.default_rng(k).integers(1, 3 * tile, k))
                n = int(sum(sizes))
                base = tg.random_trace(100 * k + variant, trace_id=k * 10 + variant, n_ranks=1, devices_per_rank=1,
                                       dev_events=n, host_events=50, n_regions=3)
                assert int(base.dev_off[1]) == n
                t = _runs_of_sizes(base, sizes, seed=k + variant)
                c.ingest([t])
                assert_trace_equal(c, t, ("run edges", shape, k, variant))
        c.reset()
    finally:
        c.close()


def test_not_sorted_hint():
    """TALP_GPU_NOT_SORTED sends every device to the sort stage without a first
    sweep: records grouped by stream (merge path), shuffled (radix path),
    already in start order (swept from their own records), and APPEND slices
    all equal the oracle; the hint with SORTED_BY_START is refused."""
    import paper_2603_26576_b300 as P
    from test_gpu_parity import _split_by_time
    c = make_ctx()
    base = tg.random_trace(31, trace_id=95, n_ranks=3, devices_per_rank=[2, 1, 3], dev_events=2500,
                           host_events=700, n_regions=3)
    for k, t in enumerate((tg.interleave_lanes(base), tg.shuffle_segments(base, seed=4), base)):
        t.trace_id = 95 + k
        c.ingest([t], flags=P.TALP_GPU_NOT_SORTED)
        assert_trace_equal(c, t, ("hint", k))
    a, b = _split_by_time(tg.interleave_lanes(base), 0.5)
    a.trace_id = b.trace_id = 99
    c.ingest([a], flags=P.TALP_GPU_NOT_SORTED)
    c.ingest([b], flags=P.TALP_GPU_NOT_SORTED | P.TALP_GPU_APPEND)
    whole = tg.Trace(**{**base.__dict__})
    whole.trace_id = 99
    assert_trace_equal(c, whole, "hint-append")
    with pytest.raises(P.TalpGpuError):
        c.ingest([base], flags=P.TALP_GPU_NOT_SORTED | P.TALP_GPU_SORTED_BY_START)
    c.close()


def test_grouped_by_stream():
    """TALP_GPU_GROUPED_BY_STREAM: each device's records grouped by stream, the
    groups found from the stream ids and merged without a first sweep: device
    and host record arrays, devices of one stream (in order already), of
    20 streams (more runs than the merge takes: the library finds them), of
    no records, a stream split into two separate stretches, and APPEND slices
    all equal the oracle; a stretch out of start order, and the flag with
    SORTED_BY_START or NOT_SORTED, are refused."""
    import torch
    import paper_2603_26576_b300 as P
    from test_gpu_parity import _split_by_time
    c = make_ctx()
    base = tg.random_trace(33, trace_id=101, n_ranks=3, devices_per_rank=[2, 1, 3], dev_events=[3000, 1, 0, 4000,
                           2500, 40000], host_events=700, n_regions=3)
    g = tg.interleave_lanes(base)
    c.ingest([g], flags=P.TALP_GPU_GROUPED_BY_STREAM)
    assert_trace_equal(c, g, "grouped, host arrays")
    dev = torch.device("cuda", 0)
    arr = {k: torch.from_numpy(getattr(g, k)).to(dev) for k in ("host_se", "host_state", "dev_se", "dev_tag")}
    g.trace_id = 102
    c.ingest([g], flags=P.TALP_GPU_GROUPED_BY_STREAM, arrays=[arr])
    assert_trace_equal(c, g, "grouped, device arrays")
    # one device of 20 streams (tags rewritten), the rest as before
    w = tg.Trace(**{**base.__dict__})
    w.dev_tag = w.dev_tag.copy()
    a0, a1 = int(w.dev_off[5]), int(w.dev_off[6])
    w.dev_tag[a0:a1] = (w.dev_tag[a0:a1] & 0xE0) | (np.arange(a1 - a0) % 20).astype(np.uint8)
    w = tg.interleave_lanes(w)
    w.trace_id = 103
    c.ingest([w], flags=P.TALP_GPU_GROUPED_BY_STREAM)
    assert_trace_equal(c, w, "grouped, 20 streams")
    # a stream in two separate stretches: still each stretch in order
    sp = tg.Trace(**{**g.__dict__})
    sp.dev_se, sp.dev_tag = g.dev_se.copy(), g.dev_tag.copy()
    b0, b1 = int(sp.dev_off[3]), int(sp.dev_off[4])
    seg_se, seg_tag = sp.dev_se[b0:b1].copy(), sp.dev_tag[b0:b1].copy()
    first = seg_tag[0] & 31
    run = np.flatnonzero((seg_tag & 31) == first)
    half = run[: len(run) // 2]
    rest = np.setdiff1d(np.arange(b1 - b0), half)
    order = np.concatenate([half, rest[(seg_tag[rest] & 31) != first], rest[(seg_tag[rest] & 31) == first]])
    sp.dev_se[b0:b1], sp.dev_tag[b0:b1] = seg_se[order], seg_tag[order]
    sp.trace_id = 104
    c.ingest([sp], flags=P.TALP_GPU_GROUPED_BY_STREAM)
    assert_trace_equal(c, sp, "grouped, a stream in two stretches")
    # APPEND slices
    a, b = _split_by_time(g, 0.5)
    a.trace_id = b.trace_id = 105
    c.ingest([a], flags=P.TALP_GPU_GROUPED_BY_STREAM)
    c.ingest([b], flags=P.TALP_GPU_GROUPED_BY_STREAM | P.TALP_GPU_APPEND)
    whole = tg.Trace(**{**base.__dict__})
    whole.trace_id = 105
    assert_trace_equal(c, whole, "grouped-append")
    # a stretch out of start order
    bad = tg.Trace(**{**g.__dict__})
    bad.dev_se = g.dev_se.copy()
    q = int(bad.dev_off[3]) + 5
    bad.dev_se[[q, q + 1]] = bad.dev_se[[q + 1, q]]
    bad.trace_id = 106
    c.ingest([bad], flags=P.TALP_GPU_GROUPED_BY_STREAM)
    st, _ = c.metrics(bad.trace_id, check=False)
    assert st == -1
    for f in (P.TALP_GPU_SORTED_BY_START, P.TALP_GPU_NOT_SORTED):
        with pytest.raises(P.TalpGpuError):
            c.ingest([g], flags=P.TALP_GPU_GROUPED_BY_STREAM | f)
    c.close()
