"""Raw activity records (per rank, all devices and streams interleaved in
delivery order) ingested through the adapter give exactly the oracle's
metrics of the same records."""
import numpy as np
import pytest

import oracle
import tracegen as tg
from gpu_common import assert_trace_equal, make_ctx

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
