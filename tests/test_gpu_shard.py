"""Sharded reduction on the GPU: a trace split by whole ranks over several
contexts (one per emulated GPU) combines, through talp_gpu_metrics_combine,
into exactly the whole trace's metrics."""
import socket

import numpy as np
import pytest

import oracle
import tracegen as tg
from gpu_common import assert_metrics_equal, make_ctx

pytestmark = pytest.mark.gpu


def _traces():
    yield tg.random_trace(21, trace_id=5, n_ranks=7, devices_per_rank=[1, 3, 0, 2, 4, 1, 2], dev_events=3000,
                          host_events=2000, n_regions=3)
    ranks, gpus, ev = tg.batched_shapes(n_traces=6, max_ranks=60, max_gpus=8, ev_lo=50, ev_hi=4000)
    t = tg.batched_trace_fast(4, ranks, gpus, ev, n_regions=8)
    t.trace_id = 6
    yield t


@pytest.mark.parametrize("world", [1, 2, 3, 4, 9])
def test_combine_of_shards_equals_whole_trace(world):
    import paper_2603_26576_b300 as P
    from paper_2603_26576_b300 import shard
    for t in _traces():
        whole_ctx = make_ctx()
        whole_ctx.ingest([t])
        whole = whole_ctx.metrics(t.trace_id)
        rec = np.diff(t.host_off.astype(np.int64))
        blocks = shard.partition_ranks(rec, world)
        ctxs, parts = [], [[] for _ in range(t.n_regions)]
        for b in blocks:
            s = shard.shard_of(t, b)
            if not s.n_ranks:
                for r in range(t.n_regions):
                    parts[r].append(dict(whole[r], **{f: 0 for f in oracle.INT_FIELDS}, n_ranks=0, m_devices=0,
                                         flags=0))
                continue
            c = make_ctx()
            c.ingest([s])
            for r, m in enumerate(c.metrics(s.trace_id)):
                parts[r].append(m)
            ctxs.append(c)
        for r in range(t.n_regions):
            got = P.metrics_to_dict(P.talp_gpu_metrics_combine(whole_ctx.ctx, parts[r]))
            assert got == whole[r], (world, t.trace_id, r)
            assert_metrics_equal(got, oracle.region_metrics(t, r), ("combined", world, r))
        for c in ctxs:
            c.close()
        whole_ctx.close()


def test_combine_rejects_mixed_parts():
    import paper_2603_26576_b300 as P
    t = next(_traces())
    c = make_ctx()
    c.ingest([t])
    m = c.metrics(t.trace_id)
    st, _ = P.talp_gpu_metrics_combine(c.ctx, [m[0], m[1]], check=False)
    assert st == -1
    st, _ = P.talp_gpu_metrics_combine(c.ctx, [], check=False)
    assert st == -1
    c.close()


def test_sharded_metrics_through_a_process_group():
    import torch.distributed as dist
    from paper_2603_26576_b300 import shard
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        t = next(_traces())
        c = make_ctx()
        got = shard.sharded_metrics(c, t)
        for r in range(t.n_regions):
            assert_metrics_equal(got[r], oracle.region_metrics(t, r), ("process-group", r))
        # the host tree with threads through the same group
        tt = tg.add_threads(t, [1 + i % 4 for i in range(t.n_ranks)], seed=2)
        po = tt.meta["proc_off"]
        got = shard.sharded_thread_metrics(c, tt, po)
        for r in range(tt.n_regions):
            want = oracle.thread_metrics(tt, r, po)
            for f in oracle.THREAD_INT_FIELDS + oracle.THREAD_RATIO_FIELDS + ("flags", "n_procs"):
                assert got[r][f] == want[f], ("process-group threads", r, f)
        c.close()
    finally:
        dist.destroy_process_group()
