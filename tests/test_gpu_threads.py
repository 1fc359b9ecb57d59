"""Host tree with threads on the GPU: every integer aggregate and ratio of
talp_gpu_thread_metrics equals the oracle's bit for bit -- tiny traces cut into
processes at random, fork-join threaded traces (processes of 1 to 100
threads, more processes than the kernel has warps), one thread per process
(equal to the GPU's own host tree of Eqs. 6-8), and the plain large trace
with 8 threads per rank at full size -- and bad process tables are refused."""
import numpy as np
import pytest

import oracle
import tracegen as tg
from gpu_common import bits, make_ctx

pytestmark = pytest.mark.gpu

INTS = ("elapsed_ns", "sum_useful", "sum_offload", "sum_busiest", "max_busiest", "n_threads")


def assert_thread_equal(g, o, tag):
    for k in INTS:
        assert g[k] == o[k], (tag, k, g[k], o[k])
    for k in oracle.THREAD_RATIO_FIELDS:
        assert bits(g[k]) == bits(o[k]), (tag, k, repr(g[k]), repr(o[k]))
    assert g["flags"] == o["flags"] and g["n_procs"] == o["n_procs"], (tag, g["flags"], o["flags"])


def check_trace(c, t, po, tag):
    res = c.thread_metrics(t.trace_id, po)
    assert len(res) == t.n_regions
    for r in range(t.n_regions):
        assert res[r]["trace_id"] == t.trace_id and res[r]["region"] == r
        assert_thread_equal(res[r], oracle.thread_metrics(t, r, po), (tag, r))
        one = c.thread_metrics(t.trace_id, po, region=r)
        assert_thread_equal(one, res[r], (tag, "single region", r))


def _groups(rng, n):
    cuts = np.sort(rng.choice(np.arange(1, n), size=int(rng.integers(0, n)), replace=False)) if n > 1 else []
    return np.concatenate([[0], cuts, [n]]).astype(np.uint32)


def test_tiny_random_processes():
    c = make_ctx()
    traces = [tg.tiny_trace(s, trace_id=s, max_ranks=7) for s in range(60)]
    c.ingest(traces)
    for s, t in enumerate(traces):
        check_trace(c, t, _groups(np.random.default_rng(s), t.n_ranks), ("tiny", s))
    c.close()


def test_one_thread_per_process_is_the_host_tree():
    c = make_ctx()
    traces = [tg.tiny_trace(s, trace_id=s) for s in range(30)]
    traces.append(tg.random_trace(5, trace_id=99, n_ranks=40, devices_per_rank=2, dev_events=300, host_events=300,
                                  n_regions=4))
    c.ingest(traces)
    pairs = (("pe", "host_pe"), ("mpi_pe", "host_mpi_pe"), ("mpi_lb", "host_mpi_lb"), ("mpi_ce", "host_mpi_ce"),
             ("oe", "host_oe"))
    for t in traces:
        th = c.thread_metrics(t.trace_id, np.arange(t.n_ranks + 1))
        host = c.metrics(t.trace_id)
        for r in range(t.n_regions):
            assert th[r]["elapsed_ns"] == host[r]["elapsed_ns"] and th[r]["thread_lb"] == 1.0
            for a, b in pairs:
                assert bits(th[r][a]) == bits(host[r][b]), (t.trace_id, r, a)
    c.close()


@pytest.mark.parametrize("threads", [[1, 4, 2], [8, 8, 8, 8], [100, 3], [33, 1, 64, 2, 31, 32]])
def test_fork_join_threads(threads):
    c = make_ctx()
    base = tg.random_trace(len(threads), trace_id=7, n_ranks=len(threads), devices_per_rank=2, dev_events=800,
                           host_events=600, n_regions=4)
    t = tg.add_threads(base, threads, seed=11)
    c.ingest([t])
    check_trace(c, t, t.meta["proc_off"], threads)
    c.close()


def test_more_processes_than_warps():
    c = make_ctx()
    base = tg.random_trace(3, trace_id=8, n_ranks=700, devices_per_rank=[1] + [0] * 699, dev_events=200,
                           host_events=30, n_regions=2)
    t = tg.add_threads(base, [1 + k % 5 for k in range(700)], seed=12)
    c.ingest([t])
    check_trace(c, t, t.meta["proc_off"], "700 processes")
    c.close()


def test_stream_ordered_variant():
    """talp_gpu_thread_metrics_device writes the same records to device memory
    without synchronising (here on a side stream)."""
    import torch
    import paper_2603_26576_b300 as P
    c = make_ctx()
    t = tg.add_threads(tg.random_trace(2, trace_id=4, n_ranks=5, dev_events=300, host_events=400, n_regions=3),
                       [3, 1, 4, 1, 5])
    po = t.meta["proc_off"]
    stream = torch.cuda.Stream()
    c.ingest([t], stream=stream.cuda_stream)
    rec = __import__("ctypes").sizeof(P.talp_gpu_thread_tree)
    out = torch.zeros(3 * rec + 8, dtype=torch.uint8, device="cuda")
    P.talp_gpu_thread_metrics_device(c.ctx, t.trace_id, P.TALP_GPU_ALL_REGIONS, po, out.data_ptr() + 8,
                                     stream.cuda_stream)
    stream.synchronize()
    got = P.thread_tree_from_bytes(out[8:].cpu().numpy().tobytes())
    assert got == c.thread_metrics(t.trace_id, po)
    for r in range(3):
        assert_thread_equal(got[r], oracle.thread_metrics(t, r, po), ("device", r))
    st = P.load_library().talp_gpu_thread_metrics_device(c.ctx, t.trace_id, 0,
                                                         np.ascontiguousarray(po).ctypes.data, len(po) - 1,
                                                         out.data_ptr() + 4, None)
    assert st == -1                                            # misaligned
    c.close()


def test_threads_across_slices_sorting_and_raw_buffers():
    """The thread tree of a trace whose device records are shuffled (the sort
    stage runs), ingested as two APPEND time slices, and of the same trace
    delivered as raw per-rank buffers, equals the oracle's on the whole trace."""
    from test_gpu_parity import _split_by_time
    c = make_ctx()
    base = tg.random_trace(21, trace_id=31, n_ranks=4, devices_per_rank=2, dev_events=3000, host_events=1500,
                           n_regions=3)
    t = tg.add_threads(base, [2, 5, 1, 3], seed=4)
    po = t.meta["proc_off"]
    sh = tg.shuffle_segments(t, seed=9)
    a, b = _split_by_time(sh, 0.5)
    c.ingest([a])
    c.ingest([b], flags=4)                                     # APPEND
    check_trace(c, t, po, "append + sort")
    raw = tg.to_raw(tg.add_threads(base, [2, 5, 1, 3], seed=4))
    raw.trace.trace_id = 32
    c.ingest_raw([raw])
    check_trace(c, raw.trace, po, "raw buffers")
    c.close()


def test_invalid_records_and_empty_regions():
    """A worker's invalid host state makes the call return EINVAL with the
    record still written and flagged; a region whose windows are empty for
    every thread is EMPTY with every ratio 1."""
    import paper_2603_26576_b300 as P
    c = make_ctx()
    t = tg.add_threads(tg.random_trace(6, trace_id=41, n_ranks=3, dev_events=200, host_events=300, n_regions=2),
                       [2, 2, 3])
    po = t.meta["proc_off"]
    bad = tg.Trace(**{**t.__dict__})
    bad.host_state = t.host_state.copy()
    bad.host_state[int(t.host_off[1]) + 3] = 3                 # a worker of process 0
    c.ingest([bad])
    st, res = P.talp_gpu_thread_metrics(c.ctx, 41, 0, po, check=False)
    assert st == -1 and res["flags"] & 0x100 and res["n_threads"] == t.n_ranks
    win = t.region_window.copy()
    win[1] = 5                                                 # region 1: [5, 5) everywhere
    empty = tg.Trace(**{**t.__dict__})
    empty.region_window = win
    c.ingest([empty])
    res = c.thread_metrics(41, po)
    assert res[1]["flags"] == 1 and res[1]["elapsed_ns"] == 0
    assert all(res[1][k] == 1.0 for k in oracle.THREAD_RATIO_FIELDS)
    for r in range(2):
        assert_thread_equal(res[r], oracle.thread_metrics(empty, r, po), ("empty", r))
    c.close()


def test_shards_of_whole_processes_combine_exactly():
    """A threaded trace split into 1-4 shards of whole processes, each reduced
    as its own trace: talp_gpu_thread_metrics_combine of the shards' records
    equals the whole trace's thread tree (and the oracle's) bit for bit."""
    import paper_2603_26576_b300 as P
    from paper_2603_26576_b300 import shard
    c = make_ctx()
    base = tg.random_trace(13, trace_id=50, n_ranks=6, devices_per_rank=2, dev_events=800, host_events=500,
                           n_regions=3)
    t = tg.add_threads(base, [3, 1, 4, 1, 5, 2], seed=6)
    po = t.meta["proc_off"].astype(np.int64)
    c.ingest([t])
    whole = c.thread_metrics(t.trace_id, po)
    for cuts in ([0, 6], [0, 2, 6], [0, 1, 4, 6], [0, 1, 2, 3, 6]):
        parts = {r: [] for r in range(t.n_regions)}
        for k in range(len(cuts) - 1):
            p0, p1 = cuts[k], cuts[k + 1]
            sh = shard.shard_of(t, np.arange(po[p0], po[p1]), trace_id=60 + k)
            c.ingest([sh])
            spo = po[p0:p1 + 1] - po[p0]
            for r, rec in enumerate(c.thread_metrics(60 + k, spo)):
                parts[r].append(dict(rec, trace_id=t.trace_id))
        for r in range(t.n_regions):
            got = P.talp_gpu_thread_metrics_combine(c.ctx, parts[r])
            assert got == whole[r], (cuts, r)
            assert_thread_equal(got, oracle.thread_metrics(t, r, po), ("combine", cuts, r))
    st, _ = P.talp_gpu_thread_metrics_combine(c.ctx, [whole[0], whole[1]], check=False)
    assert st == -1                                            # mixed regions
    c.close()


def test_bad_process_tables():
    import paper_2603_26576_b300 as P
    c = make_ctx()
    t = tg.add_threads(tg.random_trace(1, trace_id=3, n_ranks=3, dev_events=100, host_events=100, n_regions=2),
                       [2, 1, 3])
    c.ingest([t])
    n = t.n_ranks
    for po in ([1, 3, 6], [0, 3, 5], [0, 3, 3, 6], [0, 4, 2, 6], [0], [0, 6, 7]):
        st, _ = P.talp_gpu_thread_metrics(c.ctx, t.trace_id, 0, po, check=False)
        assert st == -1, po
    st, _ = P.talp_gpu_thread_metrics(c.ctx, t.trace_id, 2, [0, n], check=False)
    assert st == -1                                            # region out of range
    st, _ = P.talp_gpu_thread_metrics(c.ctx, 12345, 0, [0, n], check=False)
    assert st == -5                                            # unknown trace
    good = P.talp_gpu_thread_metrics(c.ctx, t.trace_id, 1, [0, n])
    assert_thread_equal(good, oracle.thread_metrics(t, 1, [0, n]), "one process")
    c.close()


def test_full_size_threaded_large():
    """The plain large trace (64 ranks x 4 GPUs, 576M records) with 8 threads
    per rank (213M host records more), ingested from device memory with the
    start-order flag: every region equal to the oracle."""
    import torch
    import paper_2603_26576_b300 as P
    t = tg.threaded_large()
    dev = torch.device("cuda", 0)
    arr = dict(host_se=torch.from_numpy(t.host_se).to(dev), host_state=torch.from_numpy(t.host_state).to(dev),
               dev_se=torch.from_numpy(t.dev_se).to(dev), dev_tag=torch.from_numpy(t.dev_tag).to(dev))
    c = P.Context(0)
    c.ingest([t], flags=P.TALP_GPU_SORTED_BY_START, arrays=[arr])
    res = c.thread_metrics(t.trace_id, t.meta["proc_off"])
    c.close()
    del arr
    torch.cuda.empty_cache()
    for r in range(t.n_regions):
        assert_thread_equal(res[r], oracle.thread_metrics(t, r, t.meta["proc_off"]), ("full", r))
        assert res[r]["thread_lb"] < 0.9 and res[r]["n_threads"] == 512
