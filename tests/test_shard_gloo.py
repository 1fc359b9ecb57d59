"""Multi-GPU host logic on CPU: partitioning a trace by whole ranks, slicing
its arrays, and the all-gather of region aggregates over a world-size-2
gloo group.  Shard aggregates come from the oracle here; their combination
(sums and maxima) must give the whole trace's integer aggregates exactly."""
import os
import socket

import numpy as np
import pytest

import oracle
import tracegen as tg
from oracle import INT_FIELDS
from paper_2603_26576_b300 import shard

MAX_FIELDS = ("elapsed_ns", "max_useful_offload", "max_kernel", "max_busy")


def combine_ints(parts):
    out = {}
    for f in INT_FIELDS:
        vals = [p[f] for p in parts]
        out[f] = max(vals) if f in MAX_FIELDS else sum(vals)
    out["n_ranks"] = sum(p["n_ranks"] for p in parts)
    out["m_devices"] = sum(p["m_devices"] for p in parts)
    return out


def _trace(seed=4):
    return tg.random_trace(seed, trace_id=7, n_ranks=7, devices_per_rank=[1, 3, 0, 2, 4, 1, 2], dev_events=400,
                           host_events=300, n_regions=3)


@pytest.mark.parametrize("world", [1, 2, 3, 5, 9])
def test_partition_ranks_covers_each_rank_once(world):
    rng = np.random.default_rng(world)
    for w in (rng.integers(0, 1000, 7), np.zeros(7, np.int64), np.array([5]), np.array([0, 0, 100, 0])):
        blocks = shard.partition_ranks(w, world)
        assert len(blocks) == world
        allr = np.concatenate(blocks)
        np.testing.assert_array_equal(allr, np.arange(len(w)))
        for b in blocks:
            if b.size:
                assert np.all(np.diff(b) == 1)


def test_partition_ranks_balances():
    w = np.full(64, 100)
    blocks = shard.partition_ranks(w, 4)
    assert [b.size for b in blocks] == [16, 16, 16, 16]
    w = np.array([1000] + [10] * 100)
    blocks = shard.partition_ranks(w, 2)
    assert blocks[0].tolist() == [0] and blocks[1].size == 100


def test_partition_traces_each_once_and_balanced():
    w = np.random.default_rng(3).integers(1, 10_000, 200)
    for world in (1, 2, 3, 8):
        parts = shard.partition_traces(w, world)
        np.testing.assert_array_equal(np.sort(np.concatenate(parts)), np.arange(200))
        loads = [int(w[p].sum()) for p in parts]
        assert max(loads) - min(loads) <= int(w.max())


@pytest.mark.parametrize("world", [1, 2, 3, 4, 7, 8])
def test_shard_aggregates_combine_to_whole_trace(world):
    t = _trace()
    rec = [int(t.host_off[i + 1] - t.host_off[i]) for i in range(t.n_ranks)]
    blocks = shard.partition_ranks(rec, world)
    shards = [shard.shard_of(t, b) for b in blocks]
    assert sum(s.n_records for s in shards) == t.n_records
    for r in range(t.n_regions):
        whole = oracle.region_metrics(t, r)
        parts = [oracle.region_metrics(s, r) for s in shards if s.n_ranks]
        got = combine_ints(parts)
        for f in list(INT_FIELDS) + ["n_ranks", "m_devices"]:
            assert got[f] == whole[f], (world, r, f)


def test_pack_round_trip():
    t = _trace()
    d = dict(oracle.region_metrics(t, 1), trace_id=t.trace_id, region=1)
    back = shard.unpack(shard.pack([d, d]))
    assert len(back) == 2
    from paper_2603_26576_b300 import metrics_to_dict
    assert metrics_to_dict(back[1]) == d


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = _trace()
        rec = [int(t.host_off[i + 1] - t.host_off[i]) for i in range(t.n_ranks)]
        s = shard.shard_of(t, shard.partition_ranks(rec, world)[rank])
        mine = [dict(oracle.region_metrics(s, r), trace_id=t.trace_id, region=r) for r in range(t.n_regions)]
        gathered = shard.exchange(mine)
        from paper_2603_26576_b300 import metrics_to_dict
        ok = True
        for r in range(t.n_regions):
            parts = [metrics_to_dict(x) for x in gathered[r]]
            assert [p["region"] for p in parts] == [r] * world
            got = combine_ints(parts)
            whole = oracle.region_metrics(t, r)
            ok &= all(got[f] == whole[f] for f in list(INT_FIELDS) + ["n_ranks", "m_devices"])
        q.put((rank, ok))
    finally:
        dist.destroy_process_group()


def test_exchange_world2_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
    codes = [p.exitcode for p in ps]
    assert codes == [0, 0], codes
    res = dict(q.get(timeout=5) for _ in range(2))
    assert res == {0: True, 1: True}


# ---------------------------------------------------------------- threads

THREAD_MAX = ("elapsed_ns", "max_busiest")
THREAD_SUM = ("sum_useful", "sum_offload", "sum_busiest", "n_threads", "n_procs")


def _threaded():
    return tg.add_threads(_trace(5), [3, 1, 4, 1, 5, 2, 2], seed=3)


def _combine_thread_ints(parts):
    out = {f: max(p[f] for p in parts) for f in THREAD_MAX}
    out.update({f: sum(p[f] for p in parts) for f in THREAD_SUM})
    return out


def _thread_shards(t, world):
    po = t.meta["proc_off"].astype(np.int64)
    rec = [int(t.host_off[i + 1] - t.host_off[i]) for i in range(t.n_ranks)]
    out = []
    for procs in shard.partition_processes(rec, po, world):
        if procs.size:
            out.append((shard.shard_of(t, shard.units_of(po, procs)), po[procs[0]:procs[-1] + 2] - po[procs[0]]))
    return out


@pytest.mark.parametrize("world", [1, 2, 3, 4, 7, 9])
def test_thread_shards_of_whole_processes_combine(world):
    t = _threaded()
    po = t.meta["proc_off"]
    rec = [int(t.host_off[i + 1] - t.host_off[i]) for i in range(t.n_ranks)]
    blocks = shard.partition_processes(rec, po, world)
    np.testing.assert_array_equal(np.concatenate(blocks), np.arange(len(po) - 1))
    shards = _thread_shards(t, world)
    assert sum(s.n_records for s, _ in shards) == t.n_records
    for r in range(t.n_regions):
        whole = oracle.thread_metrics(t, r, po)
        got = _combine_thread_ints([oracle.thread_metrics(s, r, spo) for s, spo in shards])
        for f in THREAD_MAX + THREAD_SUM:
            assert got[f] == whole[f], (world, r, f)


def test_pack_threads_round_trip():
    t = _threaded()
    d = dict(oracle.thread_metrics(t, 2, t.meta["proc_off"]), trace_id=t.trace_id, region=2)
    back = shard.unpack_threads(shard.pack_threads([d, d]))
    assert back == [d, d]


def _thread_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = _threaded()
        s, spo = _thread_shards(t, world)[rank]
        mine = [dict(oracle.thread_metrics(s, r, spo), trace_id=t.trace_id, region=r) for r in range(t.n_regions)]
        gathered = shard.exchange(mine, threads=True)
        ok = True
        for r in range(t.n_regions):
            assert [p["region"] for p in gathered[r]] == [r] * world
            got = _combine_thread_ints(gathered[r])
            whole = oracle.thread_metrics(t, r, t.meta["proc_off"])
            ok &= all(got[f] == whole[f] for f in THREAD_MAX + THREAD_SUM)
        q.put((rank, ok))
    finally:
        dist.destroy_process_group()


def test_thread_exchange_world2_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_thread_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
    codes = [p.exitcode for p in ps]
    assert codes == [0, 0], codes
    res = dict(q.get(timeout=5) for _ in range(2))
    assert res == {0: True, 1: True}
