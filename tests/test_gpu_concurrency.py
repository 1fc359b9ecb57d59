"""Concurrency profile on the GPU: per device, the time with at least k
active records (all kinds and kernels only), equal to the oracle bit for
bit, across chunk and tile boundaries, windows and wide timestamps."""
import numpy as np
import pytest

import oracle
import tracegen as tg
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu

EINVAL = -1


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    c.close()


def _dev(t):
    import torch
    return dict(host_se=torch.from_numpy(t.host_se).cuda(), host_state=torch.from_numpy(t.host_state).cuda(),
                dev_se=torch.from_numpy(t.dev_se).cuda(), dev_tag=torch.from_numpy(t.dev_tag).cuda())


def test_tiny_traces(ctx):
    for seed in range(150):
        t = tg.tiny_trace(seed, trace_id=seed, max_events=200)
        for r in range(t.n_regions):
            np.testing.assert_array_equal(ctx.concurrency(t, r), oracle.concurrency(t, r, 8),
                                          err_msg=str((seed, r)))


@pytest.mark.parametrize("seed", range(3))
def test_mid_size_across_chunks(ctx, seed):
    # devices longer than a chunk (16384 records) and than a tile; 4 streams
    t = tg.random_trace(seed, trace_id=seed, n_ranks=3, devices_per_rank=[2, 1, 2],
                        dev_events=[40000, 3, 0, 17000, 16384], host_events=[100, 10, 7], n_regions=4)
    arr = _dev(t)
    for r in range(t.n_regions):
        want = oracle.concurrency(t, r, 8)
        np.testing.assert_array_equal(ctx.concurrency(t, r), want, err_msg=str(("host", seed, r)))
        np.testing.assert_array_equal(ctx.concurrency(t, r, arrays=arr), want, err_msg=str(("dev", seed, r)))


@pytest.mark.parametrize("seed", range(2))
def test_high_concurrency_across_tiles_and_chunks(ctx, seed):
    """12 independent kernel streams at half occupancy each, plus copies: a
    dozen records active at once is common, so the upper half of the top-8
    lists and levels 5-8 are busy on most tiles; devices span several
    chunks and the nested windows cut tiles at both ends."""
    law = tg.DeviceLaw("lognormal", tuple(range(12)), (12, 13), occupancy=6.0)
    t = tg.random_trace(seed, trace_id=seed, n_ranks=2, devices_per_rank=[2, 1], dev_events=[40000, 17000, 999],
                        host_events=[10, 10], n_regions=4, law=law)
    arr = _dev(t)
    for r in range(t.n_regions):
        want = oracle.concurrency(t, r, 8)
        assert want[:2, 0, 7].min() > 0 and want[:2, 1, 7].min() > 0   # level 8 reached, kernels too
        np.testing.assert_array_equal(ctx.concurrency(t, r, arrays=arr), want, err_msg=str((seed, r)))


def test_long_records_running_into_later_chunks(ctx):
    """Records that start just before a chunk boundary (every 16384 records)
    or at the very start and run over many tiles of the chunks after it: the
    chunks' leading tiles are walked again with their true entering state."""
    rng = np.random.default_rng(11)
    n = 50000
    gaps = rng.integers(1, 40, n)
    s = np.cumsum(gaps).astype(np.int64)
    e = s + rng.integers(1, 60, n)
    for p, length in [(0, 10 ** 9), (16380, 300000), (16383, 50000), (32760, 200), (32767, 5_000_000),
                      (40000, 700000)]:
        e[p] = s[p] + length
    kind = rng.integers(0, 2, n).astype(np.uint8)
    kind[[16380, 32767]] = 0
    kind[16383] = 1
    base = dict(trace_id=4, n_ranks=1, devices_per_rank=np.array([1], np.uint32),
                region_window=np.array([[[0, int(e.max()) + 5]], [[int(s[20000]), int(s[45000])]]], np.int64),
                host_se=np.zeros((0, 2), np.int64), host_state=np.zeros(0, np.uint8),
                host_off=np.array([0, 0], np.uint64))
    t = tg.Trace(dev_se=np.stack([s, e], 1), dev_tag=(kind << 5).astype(np.uint8),
                 dev_off=np.array([0, n], np.uint64), **base)
    for r in range(2):
        np.testing.assert_array_equal(ctx.concurrency(t, r), oracle.concurrency(t, r, 8), err_msg=str(r))


@pytest.mark.parametrize("scale,offset", [(1 << 9, 0), (1 << 16, 0), (7, 1 << 61)])
def test_multi_chunk_wide_timestamps(ctx, scale, offset):
    """Devices of several chunks with timestamps stretched so that tiles span
    2^32 ns or more (the int64 walk, and the state kept in int64 between
    tiles), or shifted near 2^61: the main pass, the chunk scan and the
    fix-up of the chunks' leading tiles against the oracle."""
    t = tg.random_trace(5, trace_id=5, n_ranks=2, devices_per_rank=[1, 2], dev_events=[40000, 17000, 33000],
                        host_events=[10, 10], n_regions=3)
    t = tg.rescale_time(t, scale, offset)
    arr = _dev(t)
    for r in range(t.n_regions):
        np.testing.assert_array_equal(ctx.concurrency(t, r, arrays=arr), oracle.concurrency(t, r, 8),
                                      err_msg=str((scale, r)))


def test_level_one_is_the_union(ctx):
    t = tg.random_trace(7, trace_id=7, n_ranks=2, devices_per_rank=3, dev_events=30000, host_events=100,
                        n_regions=3)
    ctx.ingest([t])
    for r in range(t.n_regions):
        c = ctx.concurrency(t, r)
        _, d = ctx.unit_sums(t.trace_id, r)
        np.testing.assert_array_equal(c[:, 0, 0], d[:, 2])
        np.testing.assert_array_equal(c[:, 1, 0], d[:, 0])
    ctx.reset()


def test_wide_timestamps_and_stacked_records(ctx):
    for scale, offset in [(1 << 30, 0), (3, (1 << 61))]:
        for seed in range(20):
            t = tg.rescale_time(tg.tiny_trace(seed, trace_id=seed, max_events=300), scale, offset)
            for r in range(t.n_regions):
                np.testing.assert_array_equal(ctx.concurrency(t, r), oracle.concurrency(t, r, 8),
                                              err_msg=str((scale, seed, r)))
    # 12 identical kernels: every level saturates
    base = dict(trace_id=1, n_ranks=1, devices_per_rank=np.array([1], np.uint32),
                region_window=np.array([[[0, 10_000]]], np.int64), host_se=np.zeros((0, 2), np.int64),
                host_state=np.zeros(0, np.uint8), host_off=np.array([0, 0], np.uint64))
    t = tg.Trace(dev_se=np.array([[100, 900]] * 12, np.int64), dev_tag=np.zeros(12, np.uint8),
                 dev_off=np.array([0, 12], np.uint64), **base)
    got = ctx.concurrency(t, 0)
    assert got[0, 0].tolist() == [800] * 8 and got[0, 1].tolist() == [800] * 8


def test_errors(ctx):
    import paper_2603_26576_b300 as P
    t = tg.random_trace(3, trace_id=3, n_ranks=1, devices_per_rank=1, dev_events=20000, host_events=10)
    bad = tg.Trace(**{**t.__dict__, "dev_se": t.dev_se.copy()})
    bad.dev_se[17000, 1] = bad.dev_se[17000, 0] - 1
    st, _ = ctx.concurrency(bad, 0, check=False)
    assert st == EINVAL
    uns = tg.interleave_lanes(t)
    st, _ = ctx.concurrency(uns, 0, check=False)
    assert st == EINVAL
    b, keep = P.batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, t.host_se, t.host_state,
                                  t.host_off, t.dev_se, t.dev_tag, t.dev_off)
    st, _ = P.talp_gpu_concurrency(ctx.ctx, b, 5, check=False)
    assert st == EINVAL
    np.testing.assert_array_equal(ctx.concurrency(t, 0), oracle.concurrency(t, 0, 8))   # context still usable


def test_plain_large_tenth_all_devices(ctx):
    t = tg.plain_large(scale=0.1)
    arr = _dev(t)
    got = ctx.concurrency(t, 2, arrays=arr)
    np.testing.assert_array_equal(got, oracle.concurrency(t, 2, 8))
