"""The batched form: plans (one CUDA-graph launch over many traces) give, for
every trace and region, exactly the oracle's metrics and exactly what a
one-trace ingest gives."""
import numpy as np
import pytest

import oracle
import tracegen as tg
from gpu_common import assert_metrics_equal, make_ctx

pytestmark = pytest.mark.gpu


def _device_arrays(traces):
    import torch
    return [dict(host_se=torch.from_numpy(t.host_se).cuda(), host_state=torch.from_numpy(t.host_state).cuda(),
                 dev_se=torch.from_numpy(t.dev_se).cuda(), dev_tag=torch.from_numpy(t.dev_tag).cuda())
            for t in traces]


def _check_plan_metrics(plan, traces, tag):
    res = plan.metrics()
    assert len(res) == sum(t.n_regions for t in traces)
    q = 0
    for t in traces:
        for r in range(t.n_regions):
            assert res[q]["trace_id"] == t.trace_id and res[q]["region"] == r
            assert_metrics_equal(res[q], oracle.region_metrics(t, r), (tag, t.trace_id, r))
            q += 1


def _mixed_traces(n_tiny=200, seed0=0):
    ts = [tg.tiny_trace(s, trace_id=s, max_events=150) for s in range(seed0, seed0 + n_tiny)]
    ranks, gpus, ev = tg.batched_shapes(n_traces=40, max_ranks=24, max_gpus=4, ev_lo=5, ev_hi=3000)
    ts += [tg.batched_trace_fast(k, ranks, gpus, ev) for k in range(40)]
    for i, t in enumerate(ts):
        t.trace_id = 10_000 + i
    return ts


def test_plan_matches_oracle_and_replays():
    import torch
    c = make_ctx()
    try:
        ts = _mixed_traces()
        arrs = _device_arrays(ts)
        plan = c.plan(ts, arrs)
        info = plan.info()
        assert info["n_metrics"] == sum(t.n_regions for t in ts)
        assert info["records"] == sum(t.n_records for t in ts)
        plan.launch()
        _check_plan_metrics(plan, ts, "plan")
        plan.launch()
        plan.launch()
        _check_plan_metrics(plan, ts, "plan-replay")
        # the traces are in the context too
        one = ts[7]
        got = c.metrics(one.trace_id)
        for r in range(one.n_regions):
            assert_metrics_equal(got[r], oracle.region_metrics(one, r), ("ctx-after-plan", r))
        # new record contents at the same addresses: the next launch sees them
        k = len(ts) - 1
        t = ts[k]
        t2 = tg.Trace(**{**t.__dict__})
        t2.dev_se = t.dev_se.copy()
        t2.dev_se[:, 1] = np.maximum(t2.dev_se[:, 0], t2.dev_se[:, 1] - 500)
        arrs[k]["dev_se"].copy_(torch.from_numpy(t2.dev_se))
        torch.cuda.synchronize()
        plan.launch()
        ts[k] = t2
        _check_plan_metrics(plan, ts, "plan-new-contents")
        # a trace used by a plan cannot be reset
        import paper_2603_26576_b300 as P
        with pytest.raises(P.TalpGpuError) as ei:
            c.reset(ts[0].trace_id)
        assert ei.value.status == -6
        plan.close()
        c.reset(ts[0].trace_id)
    finally:
        c.close()


def test_plan_equals_one_trace_ingests():
    c = make_ctx()
    try:
        ts = _mixed_traces(n_tiny=30, seed0=500)
        arrs = _device_arrays(ts)
        plan = c.plan(ts, arrs)
        plan.launch()
        res = plan.metrics()
        plan.close()
        c.reset()
        q = 0
        for t, a in zip(ts, arrs):
            c.ingest([t], flags=2, arrays=[a])
            single = c.metrics(t.trace_id)
            for r in range(t.n_regions):
                assert res[q] == single[r], (t.trace_id, r)
                q += 1
    finally:
        c.close()


def test_autotuned_plan_and_unsorted_members():
    c = make_ctx()
    try:
        import paper_2603_26576_b300 as P
        ts = _mixed_traces(n_tiny=60, seed0=900)
        for i in range(0, len(ts), 3):
            ts[i] = tg.shuffle_segments(ts[i], seed=i)
        arrs = _device_arrays(ts)
        plan = c.plan(ts, arrs, flags=0, plan_flags=P.TALP_GPU_PLAN_AUTOTUNE)
        info = plan.info()
        assert info["sweep_items"] in (7, 9, 11, 13) and info["kernels_per_launch"] >= 4
        plan.launch()
        _check_plan_metrics(plan, ts, "autotuned-unsorted")
        plan.launch()
        _check_plan_metrics(plan, ts, "autotuned-unsorted-replay")
        plan.close()
    finally:
        c.close()


def test_plan_rejects_host_pointers_and_append():
    import paper_2603_26576_b300 as P
    c = make_ctx()
    try:
        t = tg.tiny_trace(1, trace_id=1)
        b, keep = P.batch_from_arrays(1, t.devices_per_rank, t.region_window, t.host_se, t.host_state, t.host_off,
                                      t.dev_se, t.dev_tag, t.dev_off)
        with pytest.raises(P.TalpGpuError) as ei:
            P.talp_gpu_plan_create(c.ctx, [b])
        assert ei.value.status == -1
    finally:
        c.close()


def test_plan_of_threaded_traces_gives_thread_trees():
    """A plan over threaded traces (one host unit per thread): after a replay
    of the graph, talp_gpu_thread_metrics of every trace equals the oracle's
    thread tree, and the plan's own results the paper's tree."""
    from gpu_common import bits
    c = make_ctx()
    try:
        ts = []
        for k in range(24):
            base = tg.random_trace(500 + k, trace_id=20_000 + k, n_ranks=1 + k % 5, devices_per_rank=1 + k % 3,
                                   dev_events=200 + 37 * k, host_events=150, n_regions=1 + k % 4)
            ts.append(tg.add_threads(base, [1 + (k + i) % 6 for i in range(base.n_ranks)], seed=k))
        plan = c.plan(ts, _device_arrays(ts))
        plan.launch()
        plan.launch()
        _check_plan_metrics(plan, ts, "threaded plan")
        for t in ts:
            po = t.meta["proc_off"]
            got = c.thread_metrics(t.trace_id, po)
            for r in range(t.n_regions):
                o = oracle.thread_metrics(t, r, po)
                for f in ("elapsed_ns", "sum_useful", "sum_offload", "sum_busiest", "max_busiest", "n_threads"):
                    assert got[r][f] == o[f], (t.trace_id, r, f)
                for f in oracle.THREAD_RATIO_FIELDS:
                    assert bits(got[r][f]) == bits(o[f]), (t.trace_id, r, f)
        plan.close()
    finally:
        c.close()
