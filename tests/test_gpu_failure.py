"""Failure path of the device-side waits, without faulting or hanging the
GPU: a context whose wait limit is negative makes every sweep report a
time-out at its first wait (a wait on a flag nothing sets).  The kernel
lets its copies in flight land, returns, and the next result call gives
ETIMEDOUT; the GPU and a fresh context stay usable."""
import pytest

import tracegen as tg
from gpu_common import assert_trace_equal, env, make_ctx

pytestmark = pytest.mark.gpu

ETIMEDOUT = -4


def test_wait_limit_runs_out_reports_etimedout():
    import paper_2603_26576_b300 as P
    t = tg.random_trace(3, trace_id=41, n_ranks=3, devices_per_rank=2, dev_events=4000, host_events=500,
                        n_regions=2)
    with env(TALP_GPU_WAIT_LIMIT=-1):
        c = P.Context(0)
    try:
        c.ingest([t], flags=P.TALP_GPU_SORTED_BY_START)
        with pytest.raises(P.TalpGpuError) as e:
            c.metrics(t.trace_id)
        assert e.value.status == ETIMEDOUT
        # the same context answers the next ingest the same way: nothing is stuck
        c.reset()
        c.ingest([t], flags=P.TALP_GPU_SORTED_BY_START)
        with pytest.raises(P.TalpGpuError) as e:
            c.metrics(t.trace_id)
        assert e.value.status == ETIMEDOUT
    finally:
        c.close()
    good = make_ctx()
    good.ingest([t], flags=P.TALP_GPU_SORTED_BY_START)
    assert_trace_equal(good, t, "after-timeout")
    good.close()


def test_wait_limit_runs_out_with_slices_handed_out():
    """The same with the sweep's dynamic work split: warps that gave up still
    take the remaining slices (writing their records empty, so the fix-up
    reads only written records); then a good context equals the oracle."""
    import paper_2603_26576_b300 as P
    t = tg.random_trace(4, trace_id=42, n_ranks=3, devices_per_rank=2, dev_events=6000, host_events=500,
                        n_regions=2)
    with env(TALP_GPU_WAIT_LIMIT=-1, TALP_GPU_SLICES_PER_WARP=16, TALP_GPU_TILES_PER_WARP=1):
        c = P.Context(0)
    try:
        for flags in (P.TALP_GPU_SORTED_BY_START, 0):
            c.ingest([t], flags=flags)
            with pytest.raises(P.TalpGpuError) as e:
                c.metrics(t.trace_id)
            assert e.value.status == ETIMEDOUT
            c.reset()
    finally:
        c.close()
    good = make_ctx(slices_per_warp=16, tiles_per_warp=1)
    good.ingest([t], flags=P.TALP_GPU_SORTED_BY_START)
    assert_trace_equal(good, t, "after-timeout, slices")
    good.close()


def test_raw_scatter_wait_runs_out_reports_etimedout():
    """The raw adapter's bounded wait for a tile's bulk copy: with a negative
    limit it reports a time-out (after letting the copy land) and the call
    returns ETIMEDOUT; a fresh context then ingests the same buffers."""
    import paper_2603_26576_b300 as P
    t = tg.random_trace(5, trace_id=43, n_ranks=2, devices_per_rank=3, dev_events=3000, host_events=300,
                        n_regions=2)
    raw = tg.to_raw(t)
    with env(TALP_GPU_WAIT_LIMIT=-1):
        c = P.Context(0)
    try:
        with pytest.raises(P.TalpGpuError) as e:
            c.ingest_raw([raw])
        assert e.value.status == ETIMEDOUT
    finally:
        c.close()
    good = make_ctx()
    good.ingest_raw([raw])
    assert_trace_equal(good, t, "raw-after-timeout", sums=False)
    good.close()
