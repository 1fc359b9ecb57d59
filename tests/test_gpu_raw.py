"""Raw activity records (per rank, all devices and streams interleaved in
delivery order) ingested through the adapter give exactly the oracle's
metrics of the same records."""
import numpy as np
import pytest

import oracle
import tracegen as tg
from gpu_common import assert_trace_equal, folded_trace, make_ctx

pytestmark = pytest.mark.gpu

EINVAL = -1


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    c.close()


def test_tiny_traces(ctx):
    ts = [tg.tiny_trace(s, trace_id=s, max_ranks=3, max_devs=3, max_events=150) for s in range(80)]
    ctx.ingest_raw([tg.to_raw(t) for t in ts])
    for t in ts:
        assert_trace_equal(ctx, t, "raw-tiny", sums=(t.trace_id % 3 == 0))
    ctx.reset()


@pytest.mark.parametrize("seed", range(3))
def test_mid_size_host_and_device_pointers(ctx, seed):
    import torch
    law = tg.DeviceLaw("lognormal", (0, 1, 2, 3), (2, 3), occupancy=0.9)
    t = tg.random_trace(seed, trace_id=50 + seed, n_ranks=3, devices_per_rank=[1, 8, 3],
                        dev_events=[9000, 3000, 1, 0, 4000, 2500, 700, 5000, 6000, 10, 2049, 4097],
                        host_events=[300, 40, 7], n_regions=3, law=law)
    r = tg.to_raw(t)
    ctx.ingest_raw([r])
    assert_trace_equal(ctx, t, ("raw-host", seed))
    ctx.reset()
    dev = dict(host_se=torch.from_numpy(t.host_se).cuda(), host_state=torch.from_numpy(t.host_state).cuda(),
               raw_se=torch.from_numpy(r.raw_se).cuda(), raw_tag=torch.from_numpy(r.raw_tag).cuda(),
               raw_dev=torch.from_numpy(r.raw_dev).cuda())
    ctx.ingest_raw([r], arrays=[dev])
    assert_trace_equal(ctx, t, ("raw-device", seed))
    ctx.reset()


def test_append_slices(ctx):
    import paper_2603_26576_b300 as P
    t = tg.random_trace(9, trace_id=77, n_ranks=2, devices_per_rank=[2, 3], dev_events=3000, host_events=500,
                        n_regions=2)
    cuts = tg.random_cuts(t, 4, seed=2)
    for k, sl in enumerate(tg.time_slices(t, cuts)):
        part = tg.Trace(trace_id=t.trace_id, n_ranks=t.n_ranks, devices_per_rank=t.devices_per_rank,
                        region_window=t.region_window, host_se=sl.host_se, host_state=sl.host_state,
                        host_off=sl.host_off, dev_se=sl.dev_se, dev_tag=sl.dev_tag, dev_off=sl.dev_off)
        ctx.ingest_raw([tg.to_raw(part)], flags=P.TALP_GPU_APPEND if k else 0)
    assert_trace_equal(ctx, t, "raw-append")
    ctx.reset()


def test_errors(ctx):
    import paper_2603_26576_b300 as P
    t = tg.random_trace(4, trace_id=5, n_ranks=2, devices_per_rank=2, dev_events=300, host_events=30)
    r = tg.to_raw(t)
    bad = tg.RawTrace(t, r.raw_se, r.raw_tag, r.raw_dev.copy(), r.raw_off)
    bad.raw_dev[17] = 2
    with pytest.raises(P.TalpGpuError) as e:
        ctx.ingest_raw([bad])
    assert e.value.status == EINVAL
    many = tg.random_trace(4, trace_id=6, n_ranks=1, devices_per_rank=9, dev_events=10, host_events=3)
    with pytest.raises(P.TalpGpuError) as e:
        ctx.ingest_raw([tg.to_raw(many)])
    assert e.value.status == EINVAL
    ctx.ingest_raw([r])                  # the context is still usable
    assert_trace_equal(ctx, t, "raw-after-errors")
    ctx.reset()


# ------------------------------------------------------------------ hold-back

def _hold_back_run(ctx, t, n_calls, seed, arrays=False):
    import torch
    import paper_2603_26576_b300 as P
    parts = tg.raw_deliveries(tg.to_raw(t), n_calls, seed=seed)
    for j, p in enumerate(parts):
        arr = None
        if arrays:
            arr = [dict(host_se=torch.from_numpy(p.trace.host_se).cuda(),
                        host_state=torch.from_numpy(p.trace.host_state).cuda(),
                        raw_se=torch.from_numpy(p.raw_se).cuda(), raw_tag=torch.from_numpy(p.raw_tag).cuda(),
                        raw_dev=torch.from_numpy(p.raw_dev).cuda())]
        ctx.ingest_raw([p], flags=P.TALP_GPU_HOLD_BACK | (P.TALP_GPU_APPEND if j else 0), arrays=arr)
        f = folded_trace(t, parts, j)
        delivered = sum(int(q.raw_off[-1]) for q in parts[:j + 1])
        assert ctx.raw_held(t.trace_id) == delivered - int(f.dev_off[-1]), ("held", seed, j)
        for r in range(t.n_regions):
            h, d = ctx.unit_sums(t.trace_id, r)
            np.testing.assert_array_equal(d, oracle.device_unions(f, r), err_msg=str(("hold", seed, j, r)))
    # flush: a call without HOLD_BACK folds every held record
    et = tg.Trace(trace_id=t.trace_id, n_ranks=t.n_ranks, devices_per_rank=t.devices_per_rank,
                  region_window=t.region_window, host_se=np.zeros((0, 2), np.int64), host_state=np.zeros(0, np.uint8),
                  host_off=np.zeros(t.n_ranks + 1, np.uint64), dev_se=np.zeros((0, 2), np.int64),
                  dev_tag=np.zeros(0, np.uint8), dev_off=np.zeros(t.m_devices + 1, np.uint64))
    empty = tg.RawTrace(et, np.zeros((0, 2), np.int64), np.zeros(0, np.uint8), np.zeros(0, np.uint8),
                        np.zeros(t.n_ranks + 1, np.uint64))
    ctx.ingest_raw([empty], flags=P.TALP_GPU_APPEND)
    assert ctx.raw_held(t.trace_id) == 0
    assert_trace_equal(ctx, t, ("hold-flush", seed))


@pytest.mark.parametrize("seed", range(4))
def test_hold_back_streamed_buffers(ctx, seed):
    law = tg.DeviceLaw("lognormal", (0, 1, 2, 3), (4, 5), occupancy=1.6)
    t = tg.random_trace(seed, trace_id=300 + seed, n_ranks=3, devices_per_rank=[2, 1, 3],
                        dev_events=[5000, 3000, 7000, 1, 0, 2600], host_events=[200, 30, 9], n_regions=3, law=law)
    _hold_back_run(ctx, t, 2 + 2 * seed, seed, arrays=(seed % 2 == 1))
    ctx.reset()


def test_hold_back_tiny_and_many_calls(ctx):
    for s in range(12):
        t = tg.tiny_trace(s, trace_id=400 + s, max_ranks=3, max_devs=3, max_events=120)
        _hold_back_run(ctx, t, 1 + s % 7, s)
    ctx.reset()


def test_hold_back_with_plain_trace_in_one_call(ctx):
    """A hold-back trace and an ordinary one in the same call, then both
    finished; the ordinary one folds at once."""
    import paper_2603_26576_b300 as P
    law = tg.DeviceLaw("lognormal", (0, 1, 2), (3,), occupancy=1.2)
    a = tg.random_trace(21, trace_id=501, n_ranks=2, devices_per_rank=2, dev_events=4000, host_events=100, law=law)
    b = tg.random_trace(22, trace_id=502, n_ranks=2, devices_per_rank=[1, 3], dev_events=2500, host_events=50)
    pa = tg.raw_deliveries(tg.to_raw(a), 3, seed=1)
    pb = tg.raw_deliveries(tg.to_raw(b), 2, seed=2)
    H, A = P.TALP_GPU_HOLD_BACK, P.TALP_GPU_APPEND
    ctx.ingest_raw([pa[0], pb[0]], flags=[H, 0])
    assert ctx.raw_held(b.trace_id) == 0
    ctx.ingest_raw([pb[1], pa[1]], flags=[A, H | A])
    ctx.ingest_raw([pa[2]], flags=A)          # last buffer, folded with the held records
    assert ctx.raw_held(a.trace_id) == 0
    assert_trace_equal(ctx, a, "hold-mixed-a")
    assert_trace_equal(ctx, b, "hold-mixed-b")
    ctx.reset()


def test_hold_back_errors(ctx):
    import paper_2603_26576_b300 as P
    t = tg.random_trace(5, trace_id=600, n_ranks=2, devices_per_rank=2, dev_events=2000, host_events=40)
    parts = tg.raw_deliveries(tg.to_raw(t), 3, seed=3)
    nomask = tg.RawTrace(parts[0].trace, parts[0].raw_se, parts[0].raw_tag, parts[0].raw_dev, parts[0].raw_off)
    with pytest.raises(P.TalpGpuError) as e:          # hold-back needs the stream masks
        ctx.ingest_raw([nomask], flags=P.TALP_GPU_HOLD_BACK)
    assert e.value.status == EINVAL
    ctx.ingest_raw([parts[0]], flags=P.TALP_GPU_HOLD_BACK)
    held = ctx.raw_held(t.trace_id)
    # a record on a stream its device does not declare: EINVAL, hold state dropped
    undeclared = parts[1].stream_mask.copy()
    i = int(np.searchsorted(parts[1].raw_off[1:], 0, side="right"))   # first rank with records
    k0 = int(parts[1].raw_off[i])
    undeclared[i, int(parts[1].raw_dev[k0])] &= ~np.uint32(1 << int(parts[1].raw_tag[k0] & 31))
    bad = tg.RawTrace(parts[1].trace, parts[1].raw_se, parts[1].raw_tag, parts[1].raw_dev, parts[1].raw_off,
                      undeclared)
    if int(parts[1].raw_off[-1]):
        with pytest.raises(P.TalpGpuError) as e:
            ctx.ingest_raw([bad], flags=P.TALP_GPU_HOLD_BACK | P.TALP_GPU_APPEND)
        assert e.value.status == EINVAL
        assert ctx.raw_held(t.trace_id) == 0
    assert held >= 0
    # shape mismatch against the held records' trace
    ctx.ingest_raw([parts[0]], flags=P.TALP_GPU_HOLD_BACK)
    other = tg.random_trace(6, trace_id=600, n_ranks=3, devices_per_rank=1, dev_events=50, host_events=5)
    op = tg.raw_deliveries(tg.to_raw(other), 2, seed=1)[1]
    with pytest.raises(P.TalpGpuError) as e:
        ctx.ingest_raw([op], flags=P.TALP_GPU_HOLD_BACK | P.TALP_GPU_APPEND)
    assert e.value.status == EINVAL
    # reset ends the hold state; the context stays usable
    ctx.reset(t.trace_id)
    assert ctx.raw_held(t.trace_id) == 0
    _hold_back_run(ctx, t, 3, 3)
    ctx.reset()


def test_many_streams_per_device(ctx):
    """Devices with up to 32 streams: more than 16 runs per lane sends the
    lanes down the sort stage's radix path; the same with hold-back, where
    every one of the 32 declared streams bounds the watermark."""
    import paper_2603_26576_b300 as P
    law = tg.DeviceLaw("lognormal", tuple(range(24)), tuple(range(24, 32)), occupancy=3.0)
    t = tg.random_trace(77, trace_id=901, n_ranks=2, devices_per_rank=[3, 2], dev_events=[6000, 9000, 1, 4000, 2049],
                        host_events=[100, 50], n_regions=2, law=law)
    assert int(np.bitwise_or.reduce(tg.stream_masks(t), axis=None)) == 0xFFFFFFFF
    ctx.ingest_raw([tg.to_raw(t)])
    assert_trace_equal(ctx, t, "raw-32-streams")
    ctx.reset()
    _hold_back_run(ctx, t, 5, 9)
    ctx.reset()


def test_device_pointers_several_traces_one_call(ctx):
    """Raw buffers of several traces in device memory, one call: every
    tile points into its own trace's arrays."""
    import torch
    ts = [tg.random_trace(90 + k, trace_id=950 + k, n_ranks=1 + k, devices_per_rank=1 + (k % 3), dev_events=1500 + 500 * k,
                          host_events=60, n_regions=2) for k in range(4)]
    rs = [tg.to_raw(t) for t in ts]
    arrays = [dict(host_se=torch.from_numpy(t.host_se).cuda(), host_state=torch.from_numpy(t.host_state).cuda(),
                   raw_se=torch.from_numpy(r.raw_se).cuda(), raw_tag=torch.from_numpy(r.raw_tag).cuda(),
                   raw_dev=torch.from_numpy(r.raw_dev).cuda()) for t, r in zip(ts, rs)]
    ctx.ingest_raw(rs, arrays=arrays)
    for t in ts:
        assert_trace_equal(ctx, t, "raw-device-multi")
    ctx.reset()


def test_hold_state_ends_with_a_new_trace_of_the_id(ctx):
    """Held records belong to their trace: an ordinary ingest of the same id
    without APPEND (a new trace) drops them, and so does reset; the new
    trace's metrics are its own."""
    import paper_2603_26576_b300 as P
    law = tg.DeviceLaw("lognormal", (0, 1, 2), (3,), occupancy=1.3)
    t = tg.random_trace(31, trace_id=970, n_ranks=2, devices_per_rank=2, dev_events=3000, host_events=100, law=law)
    parts = tg.raw_deliveries(tg.to_raw(t), 3, seed=2)
    ctx.ingest_raw([parts[0]], flags=P.TALP_GPU_HOLD_BACK)
    assert ctx.raw_held(t.trace_id) > 0
    other = tg.random_trace(32, trace_id=970, n_ranks=2, devices_per_rank=2, dev_events=800, host_events=60)
    ctx.ingest([other])
    assert ctx.raw_held(t.trace_id) == 0
    assert_trace_equal(ctx, other, "new-trace-of-the-id")
    ctx.ingest_raw([parts[0]], flags=P.TALP_GPU_HOLD_BACK)
    assert ctx.raw_held(t.trace_id) > 0
    ctx.reset(t.trace_id)
    assert ctx.raw_held(t.trace_id) == 0
    _hold_back_run(ctx, t, 3, 2)
    ctx.reset()


def test_streams_that_do_not_interleave(ctx):
    """Devices whose lane is several streams are sorted without a first
    sweep; here some of them are already in start order (streams one after
    the other in time, or every record starting at the same time) and are
    swept from their own records, others interleave and are merged.  Every
    unit equals the oracle."""
    rng = np.random.default_rng(8)
    segs = []
    for kind in ("phases", "interleaved", "same_start", "one_stream", "phases", "empty"):
        if kind == "empty":
            segs.append((np.zeros((0, 2), np.int64), np.zeros(0, np.uint8)))
            continue
        n = 600
        if kind == "phases":          # stream 0, then stream 1, then stream 2, in time
            s = np.sort(rng.integers(0, 30_000, n))
            st = np.minimum(np.arange(n) * 3 // n, 2)
        elif kind == "interleaved":
            s = np.sort(rng.integers(0, 30_000, n))
            st = rng.integers(0, 3, n)
        elif kind == "same_start":
            s = np.full(n, 777)
            st = rng.integers(0, 2, n)
        else:
            s = np.sort(rng.integers(0, 30_000, n))
            st = np.zeros(n, np.int64)
        d = rng.integers(1, 400, n)
        se = np.stack([s, s + d], axis=1).astype(np.int64)
        kd = rng.choice(np.array([0, 0, 0, 1, 2], np.uint8), n)
        segs.append((se, tg.make_tag(kd, st.astype(np.uint8))))
    dpr = np.array([3, 3], np.uint32)
    dev_off = np.concatenate([[0], np.cumsum([x[0].shape[0] for x in segs])]).astype(np.uint64)
    host = [np.array([[0, 12_000], [12_000, 31_000]], np.int64), np.array([[0, 31_000]], np.int64)]
    t = tg.Trace(trace_id=90, n_ranks=2, devices_per_rank=dpr,
                 region_window=np.array([[[0, 31_000], [0, 31_000]], [[5_000, 20_000], [100, 900]]], np.int64),
                 host_se=np.concatenate(host), host_state=np.array([0, 1, 2], np.uint8),
                 host_off=np.array([0, 2, 3], np.uint64), dev_se=np.concatenate([x[0] for x in segs]),
                 dev_tag=np.concatenate([x[1] for x in segs]), dev_off=dev_off)
    raw = tg.to_raw(t)
    ctx.ingest_raw([raw])
    assert_trace_equal(ctx, t, "streams-in-order")
    ctx.reset()


@pytest.mark.parametrize("n_events", [300, 40_000])
def test_stream_out_of_start_order_is_reported(ctx, n_events):
    """A raw buffer must deliver each stream in start order (a stream
    executes in order).  The adapter takes each device lane's streams as its
    sorted runs, so a stream delivered out of order is reported by the next
    result call (EINVAL), whether the descent falls inside a chunk of the
    merge or across two; the same buffer in order is exact."""
    import paper_2603_26576_b300 as P
    t = tg.random_trace(12, trace_id=77, n_ranks=1, devices_per_rank=1, dev_events=n_events, host_events=50)
    # three streams on the one device, interleaved in time
    tag = (t.dev_tag & 0xE0) | (np.arange(t.n_dev) % 3).astype(np.uint8)
    t = tg.Trace(trace_id=77, n_ranks=1, devices_per_rank=t.devices_per_rank, region_window=t.region_window,
                 host_se=t.host_se, host_state=t.host_state, host_off=t.host_off, dev_se=t.dev_se, dev_tag=tag,
                 dev_off=t.dev_off)
    r = tg.to_raw(t)
    ctx.ingest_raw([r])
    assert_trace_equal(ctx, t, "raw-in-order", sums=False)
    ctx.reset()
    # swap two records of one stream with different starts: the stream's
    # delivery is no longer in start order
    se = r.raw_se.copy()
    st = r.raw_tag & 31
    idx = np.flatnonzero(st == 1)
    a, b = int(idx[len(idx) // 3]), int(idx[len(idx) // 3 + 1])
    assert se[a, 0] < se[b, 0]
    se[[a, b]] = se[[b, a]]
    bad = tg.RawTrace(t, se, r.raw_tag, r.raw_dev, r.raw_off)
    ctx.ingest_raw([bad])
    with pytest.raises(P.TalpGpuError) as e:
        ctx.metrics(77)
    assert e.value.status == EINVAL
    ctx.reset()
