"""The served form: jobs stream time slices into device-resident running
state while clients query it.  Every answer must equal the oracle on the
records submitted so far (bit-exact), whatever else the server is doing."""
import threading

import numpy as np
import pytest

import oracle
import tracegen as tg
from gpu_common import assert_metrics_equal, folded_trace, make_ctx

pytestmark = pytest.mark.gpu

EINVAL, ENOMEM, ENOTFOUND, EBUSY = -1, -2, -5, -6


def _jobs(seed0=0):
    ts = [tg.tiny_trace(s, trace_id=100 + s, max_events=200) for s in range(seed0, seed0 + 6)]
    ts += [tg.random_trace(seed0 + 7, trace_id=200, n_ranks=3, devices_per_rank=2, dev_events=4000,
                           host_events=2500)]
    ranks, gpus, ev = tg.batched_shapes(n_traces=12, max_ranks=40, max_gpus=4, ev_lo=20, ev_hi=3000)
    for k in range(12):
        t = tg.batched_trace_fast(k, ranks, gpus, ev, n_regions=4)
        t.trace_id = 300 + k
        ts.append(t)
    return ts


def _submit(srv, t, sl):
    return srv.submit(t.trace_id, sl.host_se, sl.host_state, sl.host_off, sl.dev_se, sl.dev_tag, sl.dev_off,
                      sorted_by_start=sl.sorted_by_start)


def _client(srv, t, slices, results, errors):
    try:
        results.append(srv.query(t.trace_id))          # nothing folded yet
        for sl in slices:
            _submit(srv, t, sl)
            results.append(srv.query(t.trace_id))
    except Exception as e:  # pragma: no cover - reported by the test
        errors.append((t.trace_id, repr(e)))


def _check_prefixes(t, cuts, results, tag):
    assert len(results) == cuts.shape[0] + 2
    for k, res in enumerate(results):
        p = tg.prefix_trace(t, cuts, k - 1)
        for r in range(t.n_regions):
            assert_metrics_equal(res[r], oracle.region_metrics(p, r), (tag, t.trace_id, "slices", k, r))


def test_serving_prefix_parity_concurrent_clients():
    from paper_2603_26576_b300 import Server
    c = make_ctx()
    ts = _jobs()
    with Server(c, max_jobs=64, max_slice_records=1 << 18, staging_slices=16) as srv:
        plan = []
        for i, t in enumerate(ts):
            cuts = tg.random_cuts(t, 3 + i % 4, seed=11)
            slices = tg.time_slices(t, cuts, shuffle_seed=(7 if i % 3 == 0 else None))
            srv.open_job(t.trace_id, t.devices_per_rank, t.region_window)
            plan.append((t, cuts, slices, []))
        errors = []
        th = [threading.Thread(target=_client, args=(srv, t, sl, res, errors)) for t, _, sl, res in plan]
        for x in th:
            x.start()
        for x in th:
            x.join()
        assert not errors, errors
        srv.drain()
        st = srv.stats()
        assert st["slices_submitted"] == st["slices_folded"] == sum(len(p[2]) for p in plan)
        assert st["records_folded"] == sum(t.n_records for t in ts)
        assert st["queries"] == sum(len(p[3]) for p in plan)
        assert st["jobs_open"] == len(ts)
        assert 0 < st["query_p50_ms"] <= st["query_p99_ms"] <= st["query_max_ms"]
    for t, cuts, _, res in plan:
        _check_prefixes(t, cuts, res, "served")
    c.close()


def test_serving_alone_equals_mixed_equals_plain():
    from paper_2603_26576_b300 import Server
    c = make_ctx()
    ts = _jobs(seed0=40)
    x = ts[6]
    cuts = tg.random_cuts(x, 5, seed=3)
    slices = tg.time_slices(x, cuts, shuffle_seed=2)
    # alone
    with Server(c, max_jobs=64, max_slice_records=1 << 18) as srv:
        srv.open_job(x.trace_id, x.devices_per_rank, x.region_window)
        for sl in slices:
            _submit(srv, x, sl)
        alone = srv.query(x.trace_id)
    # in a mix of concurrently streaming jobs
    with Server(c, max_jobs=64, max_slice_records=1 << 18) as srv:
        plan = []
        for t in ts:
            ct = tg.random_cuts(t, 4, seed=9) if t is not x else cuts
            sl = tg.time_slices(t, ct, shuffle_seed=4) if t is not x else slices
            srv.open_job(t.trace_id, t.devices_per_rank, t.region_window)
            plan.append((t, sl, []))
        errors = []
        th = [threading.Thread(target=_client, args=(srv, t, sl, res, errors)) for t, sl, res in plan]
        for h in th:
            h.start()
        for h in th:
            h.join()
        assert not errors, errors
        mixed = [p for p in plan if p[0] is x][0][2][-1]
    # one plain ingest of the whole trace
    c.ingest([x], flags=0)
    plain = c.metrics(x.trace_id)
    c.reset()
    for r in range(x.n_regions):
        assert alone[r] == mixed[r], ("alone-vs-mixed", r)
        assert alone[r] == plain[r], ("alone-vs-plain", r)
        assert_metrics_equal(alone[r], oracle.region_metrics(x, r), ("served-full", r))
    c.close()


def test_serving_admission_slots_and_budget():
    from paper_2603_26576_b300 import Server
    small = tg.tiny_trace(3, trace_id=1, max_events=50)
    c = make_ctx(budget=8 << 20)
    with Server(c, max_jobs=2, max_slice_records=4096, staging_slices=4) as srv:
        assert srv.open_job(1, small.devices_per_rank, small.region_window) == 0
        assert srv.open_job(2, small.devices_per_rank, small.region_window) == 0
        assert srv.open_job(3, small.devices_per_rank, small.region_window, check=False) == EBUSY
        assert srv.open_job(2, small.devices_per_rank, small.region_window, check=False) == EBUSY
        srv.close_job(2)
        # a job whose running state alone exceeds what the budget leaves
        n = 20000
        win = np.zeros((8, n, 2), np.int64)
        win[:, :, 1] = 1000
        assert srv.open_job(4, np.ones(n, np.uint32), win, check=False) == ENOMEM
        assert srv.stats()["jobs_open"] == 1
        # the server is still serving the admitted job
        cuts = tg.random_cuts(small, 2, seed=1)
        for sl in tg.time_slices(small, cuts):
            srv.submit(1, sl.host_se, sl.host_state, sl.host_off, sl.dev_se, sl.dev_tag, sl.dev_off)
        res = srv.query(1)
        for r in range(small.n_regions):
            assert_metrics_equal(res[r], oracle.region_metrics(small, r), ("after-admission", r))
        assert srv.open_job(5, small.devices_per_rank, small.region_window) == 0
    c.close()


def test_serving_errors_stay_with_their_job():
    from paper_2603_26576_b300 import Server, talp_gpu_server_query
    c = make_ctx()
    good = tg.tiny_trace(11, trace_id=21, max_events=120)
    bad = tg.random_trace(12, trace_id=22, n_ranks=2, devices_per_rank=1, dev_events=300, host_events=200)
    with Server(c, max_jobs=8, max_slice_records=4096) as srv:
        for t in (good, bad):
            srv.open_job(t.trace_id, t.devices_per_rank, t.region_window)
        # argument errors are refused at submit
        hoff = bad.host_off.copy()
        hoff[1] = hoff[2] + 1
        assert srv.submit(bad.trace_id, bad.host_se, bad.host_state, hoff, bad.dev_se, bad.dev_tag,
                          bad.dev_off, check=False) == EINVAL
        assert srv.submit(999, good.host_se, good.host_state, good.host_off, good.dev_se, good.dev_tag,
                          good.dev_off, check=False) == ENOTFOUND
        n = 5000
        off = np.zeros(good.n_ranks + 1, np.uint64)
        off[1:] = n
        assert srv.submit(good.trace_id, np.zeros((n, 2), np.int64), np.zeros(n, np.uint8), off, good.dev_se,
                          good.dev_tag, good.dev_off, check=False) == EINVAL
        # a record with end < start makes its own job's metrics invalid only
        dse = bad.dev_se.copy()
        dse[0, 1] = dse[0, 0] - 1
        srv.submit(good.trace_id, good.host_se, good.host_state, good.host_off, good.dev_se, good.dev_tag,
                   good.dev_off)
        srv.submit(bad.trace_id, bad.host_se, bad.host_state, bad.host_off, dse, bad.dev_tag, bad.dev_off)
        st, _ = srv.query(bad.trace_id, check=False)
        assert st == EINVAL
        res = srv.query(good.trace_id)
        for r in range(good.n_regions):
            assert_metrics_equal(res[r], oracle.region_metrics(good, r), ("good-beside-bad", r))
        st, _ = talp_gpu_server_query(srv.handle, 999, 0, check=False)
        assert st == ENOTFOUND
        st, _ = talp_gpu_server_query(srv.handle, good.trace_id, good.n_regions, check=False)
        assert st == EINVAL
    c.close()


# ------------------------------------------------------- raw activity buffers

def _raw_client(srv, t, parts, results, errors):
    try:
        for p in parts:
            srv.submit_raw(t.trace_id, p.trace.host_se, p.trace.host_state, p.trace.host_off, p.raw_se, p.raw_tag,
                           p.raw_dev, p.raw_off, stream_mask=p.stream_mask, hold_back=True)
            results.append(srv.query(t.trace_id))
        z = np.zeros(t.n_ranks + 1, np.uint64)
        srv.submit_raw(t.trace_id, np.zeros((0, 2), np.int64), np.zeros(0, np.uint8), z, np.zeros((0, 2), np.int64),
                       np.zeros(0, np.uint8), np.zeros(0, np.uint8), z, hold_back=False)   # flush
        results.append(srv.query(t.trace_id))
    except Exception as e:  # pragma: no cover - reported by the test
        errors.append((t.trace_id, repr(e)))


def test_serving_raw_buffers_hold_back():
    """Jobs stream raw activity buffers (streams interleaved in completion
    order) with hold-back; every answer equals the oracle on the records
    folded so far (per device, those at or before the watermark), and after
    the flush on the whole trace."""
    from paper_2603_26576_b300 import Server
    c = make_ctx()
    law = tg.DeviceLaw("lognormal", (0, 1, 2, 3), (4, 5), occupancy=1.5)
    ts = [tg.random_trace(40 + k, trace_id=700 + k, n_ranks=2 + k % 3, devices_per_rank=1 + k % 4,
                          dev_events=1500 + 700 * k, host_events=200, n_regions=3, law=law) for k in range(6)]
    ts += [tg.tiny_trace(s, trace_id=720 + s, max_ranks=3, max_devs=3, max_events=150) for s in range(6)]
    with Server(c, max_jobs=32, max_slice_records=1 << 17, staging_slices=8) as srv:
        plan = []
        for i, t in enumerate(ts):
            parts = tg.raw_deliveries(tg.to_raw(t), 2 + i % 5, seed=i)
            srv.open_job(t.trace_id, t.devices_per_rank, t.region_window)
            plan.append((t, parts, [], []))
        th = [threading.Thread(target=_raw_client, args=(srv, t, parts, res, err)) for t, parts, res, err in plan]
        for x in th:
            x.start()
        for x in th:
            x.join()
        for t, parts, res, err in plan:
            assert not err, err
            assert len(res) == len(parts) + 1
            for j in range(len(parts)):
                f = folded_trace(t, parts, j)
                for r in range(t.n_regions):
                    assert_metrics_equal(res[j][r], oracle.region_metrics(f, r), ("raw-serve", t.trace_id, j, r))
            for r in range(t.n_regions):
                assert_metrics_equal(res[-1][r], oracle.region_metrics(t, r), ("raw-serve-flush", t.trace_id, r))
            srv.close_job(t.trace_id)
        st = srv.stats()
        assert st["jobs_open"] == 0
    c.close()


def test_serving_raw_bad_buffer_stays_with_its_submitter():
    """A raw buffer with a record on a stream its device never declared, or
    naming a device its rank lacks, is refused at submission (EINVAL) and
    nothing of it is queued; the jobs' other raw buffers, folded in the same
    waves, give the oracle's metrics of their whole traces."""
    from paper_2603_26576_b300 import Server
    c = make_ctx()
    law = tg.DeviceLaw("lognormal", (0, 1, 2), (3, 4), occupancy=1.2)
    good = tg.random_trace(61, trace_id=801, n_ranks=2, devices_per_rank=2, dev_events=2000, host_events=100, law=law)
    bad = tg.random_trace(62, trace_id=802, n_ranks=2, devices_per_rank=[1, 2], dev_events=1500, host_events=80,
                          law=law)
    pg = tg.raw_deliveries(tg.to_raw(good), 3, seed=4)
    pb = tg.raw_deliveries(tg.to_raw(bad), 3, seed=5)
    with Server(c, max_jobs=8, max_slice_records=1 << 16, staging_slices=4) as srv:
        for t in (good, bad):
            srv.open_job(t.trace_id, t.devices_per_rank, t.region_window)

        def sub(t, p, tag=None, dev=None, hold=True, check=True):
            return srv.submit_raw(t.trace_id, p.trace.host_se, p.trace.host_state, p.trace.host_off, p.raw_se,
                                  p.raw_tag if tag is None else tag, p.raw_dev if dev is None else dev, p.raw_off,
                                  stream_mask=p.stream_mask, hold_back=hold, check=check)
        sub(good, pg[0])
        sub(bad, pb[0])
        assert int(pb[1].raw_off[1]) > 0, "rank 0 of the second buffer has records"
        tag = pb[1].raw_tag.copy()
        tag[0] = (tag[0] & 0xE0) | 31                    # stream 31: never declared
        assert sub(bad, pb[1], tag=tag, check=False) == EINVAL
        dev = pb[1].raw_dev.copy()
        dev[0] = 1                                       # rank 0 has one device
        assert sub(bad, pb[1], dev=dev, check=False) == EINVAL
        sub(good, pg[1])
        sub(bad, pb[1])
        sub(good, pg[2], hold=False)
        sub(bad, pb[2], hold=False)
        for t in (good, bad):
            res = srv.query(t.trace_id)
            for r in range(t.n_regions):
                assert_metrics_equal(res[r], oracle.region_metrics(t, r), ("raw-bad-buffer", t.trace_id, r))
    c.close()


def test_serving_raw_job_closed_with_held_records_reopens_clean():
    """Closing a job drops its held raw records with its state; the same id
    opened again starts from nothing."""
    from paper_2603_26576_b300 import Server
    c = make_ctx()
    law = tg.DeviceLaw("lognormal", (0, 1, 2), (3,), occupancy=1.3)
    t = tg.random_trace(71, trace_id=880, n_ranks=2, devices_per_rank=2, dev_events=2500, host_events=90, law=law)
    parts = tg.raw_deliveries(tg.to_raw(t), 3, seed=6)
    with Server(c, max_jobs=4, max_slice_records=1 << 16, staging_slices=4) as srv:
        def sub(p, hold=True):
            srv.submit_raw(t.trace_id, p.trace.host_se, p.trace.host_state, p.trace.host_off, p.raw_se, p.raw_tag,
                           p.raw_dev, p.raw_off, stream_mask=p.stream_mask, hold_back=hold)
        srv.open_job(t.trace_id, t.devices_per_rank, t.region_window)
        sub(parts[0])
        sub(parts[1])
        srv.query(t.trace_id)                  # both folded (with whatever they hold back)
        assert c.raw_held(t.trace_id) > 0
        srv.close_job(t.trace_id)
        assert c.raw_held(t.trace_id) == 0
        srv.open_job(t.trace_id, t.devices_per_rank, t.region_window)
        for j, p in enumerate(parts):
            sub(p, hold=j < len(parts) - 1)
        res = srv.query(t.trace_id)
        for r in range(t.n_regions):
            assert_metrics_equal(res[r], oracle.region_metrics(t, r), ("reopened", r))
    c.close()


def test_served_thread_tree_prefixes_mixed_with_metrics_queries():
    """Jobs of threaded traces: after every slice a client asks for the host
    tree with threads and another for the paper's metrics, concurrently; the
    thread answers (batched with the metrics queries on the query stream)
    equal the oracle's thread tree on the submitted prefix, bit for bit.  A
    bad process table is refused at the call."""
    from gpu_common import bits
    from paper_2603_26576_b300 import Server
    c = make_ctx()
    jobs = []
    for k, T in enumerate(([2, 3, 1], [4, 4], [1, 1, 1, 1], [5, 2, 7])):
        base = tg.random_trace(60 + k, trace_id=700 + k, n_ranks=len(T), devices_per_rank=2, dev_events=1500,
                               host_events=800, n_regions=3)
        jobs.append(tg.add_threads(base, T, seed=k))
    with Server(c, max_jobs=16, max_slice_records=1 << 18, staging_slices=16) as srv:
        plan = []
        for i, t in enumerate(jobs):
            cuts = tg.random_cuts(t, 3 + i % 3, seed=13)
            slices = tg.time_slices(t, cuts, shuffle_seed=(5 if i % 2 else None))
            srv.open_job(t.trace_id, t.devices_per_rank, t.region_window)
            plan.append((t, cuts, slices, [], []))
        errors = []

        def thread_client(t, slices, tres, mres):
            try:
                po = t.meta["proc_off"]
                tres.append(srv.query_threads(t.trace_id, po))
                for sl in slices:
                    _submit(srv, t, sl)
                    tres.append(srv.query_threads(t.trace_id, po))
                    mres.append(srv.query(t.trace_id, region=1))
            except Exception as e:  # pragma: no cover - reported by the test
                errors.append((t.trace_id, repr(e)))

        th = [threading.Thread(target=thread_client, args=(t, sl, tr, mr)) for t, _, sl, tr, mr in plan]
        for x in th:
            x.start()
        for x in th:
            x.join()
        assert not errors, errors
        t0 = jobs[0]
        st, _ = srv.query_threads(t0.trace_id, [0, 2, 2, t0.n_ranks], check=False)
        assert st == EINVAL
        st, _ = srv.query_threads(t0.trace_id, [0, t0.n_ranks + 1], check=False)
        assert st == EINVAL
    for t, cuts, _, tres, mres in plan:
        po = t.meta["proc_off"]
        assert len(tres) == cuts.shape[0] + 2
        for k, res in enumerate(tres):
            p = tg.prefix_trace(t, cuts, k - 1)
            for r in range(t.n_regions):
                o = oracle.thread_metrics(p, r, po)
                for f in ("elapsed_ns", "sum_useful", "sum_offload", "sum_busiest", "max_busiest", "n_threads"):
                    assert res[r][f] == o[f], (t.trace_id, k, r, f)
                for f in oracle.THREAD_RATIO_FIELDS:
                    assert bits(res[r][f]) == bits(o[f]), (t.trace_id, k, r, f)
        for k, m in enumerate(mres):
            assert_metrics_equal(m, oracle.region_metrics(tg.prefix_trace(t, cuts, k), 1), (t.trace_id, k))
    c.close()
