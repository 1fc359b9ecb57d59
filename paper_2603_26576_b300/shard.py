"""Multi-GPU form of the reduction: host logic only (argument marshalling and
the exchange of per-shard aggregates; every step of the computation runs in
the CUDA library).

A trace's units are independent: a rank's host intervals and each of its
devices' records are reduced on their own (Sec. 4.1, 4.2), and the region's
metrics need only sums and maxima over units (Eqs. 1, 6-12).  A trace is
therefore split by whole ranks (each rank with all of its devices, so no
device segment and no carry crosses GPUs); each GPU reduces its shard to the
region aggregates (one talp_gpu_metrics record per region, 184 bytes), the
records are all-gathered, and talp_gpu_metrics_combine forms the ratios of
the whole trace.  Independent traces (the batched form) are split by whole
traces with no exchange at all.  The host tree with threads splits by whole
processes (each with all of its threads and their devices) and exchanges
talp_gpu_thread_tree records (112 bytes) the same way.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib

RECORD_BYTES = ctypes.sizeof(_lib.talp_gpu_metrics)
THREAD_RECORD_BYTES = ctypes.sizeof(_lib.talp_gpu_thread_tree)


def partition_ranks(records_per_rank, world: int) -> list:
    """Contiguous blocks of ranks, one per GPU, balanced by record count:
    block k ends at the first rank whose prefix count reaches k/world of the
    total.  Every rank is in exactly one block; a block may be empty only
    when there are fewer ranks than GPUs."""
    w = np.asarray(records_per_rank, np.float64)
    n = w.shape[0]
    if world < 1:
        raise ValueError("world must be >= 1")
    cum = np.concatenate([[0.0], np.cumsum(w)])
    total = cum[-1]
    cuts = [0]
    for k in range(1, world):
        if total > 0:
            c = int(np.searchsorted(cum, total * k / world, side="left"))
        else:
            c = (n * k) // world
        cuts.append(min(max(c, cuts[-1]), n))
    cuts.append(n)
    # ranks left over by ties go to the empty blocks at the end
    return [np.arange(cuts[k], cuts[k + 1], dtype=np.int64) for k in range(world)]


def partition_processes(records_per_unit, proc_off, world: int) -> list:
    """Contiguous blocks of whole processes (proc_off groups the host units),
    balanced by record count as partition_ranks does; returns per GPU the
    block's process indices."""
    po = np.asarray(proc_off, np.int64)
    w = np.asarray(records_per_unit, np.float64)
    cum = np.concatenate([[0.0], np.cumsum(w)])
    per_proc = cum[po[1:]] - cum[po[:-1]]
    return partition_ranks(per_proc, world)


def units_of(proc_off, procs) -> np.ndarray:
    """Host units (threads) of a contiguous block of processes."""
    po = np.asarray(proc_off, np.int64)
    procs = np.asarray(procs, np.int64)
    if procs.size == 0:
        return np.zeros(0, np.int64)
    return np.arange(po[procs[0]], po[procs[-1] + 1], dtype=np.int64)


def partition_traces(records_per_trace, world: int) -> list:
    """Whole traces to GPUs, longest first onto the least loaded GPU."""
    w = np.asarray(records_per_trace, np.int64)
    load = np.zeros(world, np.int64)
    out = [[] for _ in range(world)]
    for k in np.argsort(-w, kind="stable"):
        g = int(np.argmin(load))
        out[g].append(int(k))
        load[g] += w[k]
    return [np.array(sorted(x), np.int64) for x in out]


@dataclass
class Shard:
    """The sub-trace of a block of ranks (same attribute names as a trace)."""
    trace_id: int
    n_ranks: int
    devices_per_rank: np.ndarray
    region_window: np.ndarray
    host_se: np.ndarray
    host_state: np.ndarray
    host_off: np.ndarray
    dev_se: np.ndarray
    dev_tag: np.ndarray
    dev_off: np.ndarray
    ranks: np.ndarray

    @property
    def n_regions(self) -> int:
        return int(self.region_window.shape[0])

    @property
    def n_records(self) -> int:
        return int(self.host_se.shape[0] + self.dev_se.shape[0])


def shard_of(t, ranks, trace_id=None) -> Shard:
    """Slice the CSR arrays of trace `t` down to the contiguous block `ranks`."""
    ranks = np.asarray(ranks, np.int64)
    dpr = np.asarray(t.devices_per_rank, np.uint32)
    hoff = np.asarray(t.host_off, np.uint64)
    doff = np.asarray(t.dev_off, np.uint64)
    if ranks.size and np.any(np.diff(ranks) != 1):
        raise ValueError("a shard is a contiguous block of ranks")
    r0 = int(ranks[0]) if ranks.size else 0
    r1 = int(ranks[-1]) + 1 if ranks.size else 0
    dstart = np.concatenate([[0], np.cumsum(dpr.astype(np.int64))])
    g0, g1 = int(dstart[r0]), int(dstart[r1])
    h0, h1 = int(hoff[r0]), int(hoff[r1])
    d0, d1 = int(doff[g0]), int(doff[g1])
    return Shard(trace_id=int(t.trace_id if trace_id is None else trace_id), n_ranks=r1 - r0,
                 devices_per_rank=np.ascontiguousarray(dpr[r0:r1]),
                 region_window=np.ascontiguousarray(np.asarray(t.region_window)[:, r0:r1]),
                 host_se=np.ascontiguousarray(t.host_se[h0:h1]), host_state=np.ascontiguousarray(t.host_state[h0:h1]),
                 host_off=(hoff[r0:r1 + 1] - hoff[r0]).astype(np.uint64),
                 dev_se=np.ascontiguousarray(t.dev_se[d0:d1]), dev_tag=np.ascontiguousarray(t.dev_tag[d0:d1]),
                 dev_off=(doff[g0:g1 + 1] - doff[g0]).astype(np.uint64), ranks=ranks)


def pack(records) -> np.ndarray:
    """talp_gpu_metrics records (structs or dicts) -> uint8[k, RECORD_BYTES]."""
    out = np.zeros((len(records), RECORD_BYTES), np.uint8)
    for k, r in enumerate(records):
        s = r if isinstance(r, _lib.talp_gpu_metrics) else _lib.metrics_from_dict(r)
        out[k] = np.frombuffer(bytes(s), np.uint8)
    return out


def unpack(buf) -> list:
    buf = np.ascontiguousarray(buf, np.uint8).reshape(-1, RECORD_BYTES)
    return [_lib.talp_gpu_metrics.from_buffer_copy(buf[k].tobytes()) for k in range(buf.shape[0])]


def pack_threads(records) -> np.ndarray:
    """talp_gpu_thread_tree records (structs or dicts) -> uint8[k, THREAD_RECORD_BYTES]."""
    out = np.zeros((len(records), THREAD_RECORD_BYTES), np.uint8)
    for k, r in enumerate(records):
        if not isinstance(r, _lib.talp_gpu_thread_tree):
            x = _lib.talp_gpu_thread_tree()
            for f, _ in _lib.talp_gpu_thread_tree._fields_:
                setattr(x, f, r[f])
            r = x
        out[k] = np.frombuffer(bytes(r), np.uint8)
    return out


def unpack_threads(buf) -> list:
    """uint8[k, THREAD_RECORD_BYTES] -> thread-tree records as dicts."""
    return _lib.thread_tree_from_bytes(np.ascontiguousarray(buf, np.uint8).tobytes())


def exchange(records, group=None, threads=False) -> list:
    """All-gather the region records of every rank of the process group:
    returns, per region, the list of records of all ranks (rank order).
    talp_gpu_metrics records, or thread-tree records with threads=True.
    Works on gloo (CPU tensors) and nccl (CUDA tensors)."""
    import torch
    import torch.distributed as dist
    local = torch.from_numpy(pack_threads(records) if threads else pack(records))
    if dist.get_backend(group) == "nccl":
        local = local.cuda()
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(bufs, local, group=group)
    per_rank = [(unpack_threads if threads else unpack)(b.cpu().numpy()) for b in bufs]
    return [[per_rank[w][r] for w in range(world)] for r in range(len(records))]


def sharded_metrics(ctx, t, group=None, stream=None) -> list:
    """Metrics of every region of trace `t` reduced across the ranks of the
    process group: this process ingests its block of ranks into `ctx`
    (its GPU), exchanges the region aggregates and combines them."""
    import torch.distributed as dist
    world, me = dist.get_world_size(group), dist.get_rank(group)
    hoff = np.asarray(t.host_off, np.int64)
    doff = np.asarray(t.dev_off, np.int64)
    dstart = np.concatenate([[0], np.cumsum(np.asarray(t.devices_per_rank, np.int64))])
    rec = np.diff(hoff) + (doff[dstart[1:]] - doff[dstart[:-1]])
    block = partition_ranks(rec, world)[me]
    s = shard_of(t, block)
    R = s.n_regions
    if s.n_ranks:
        ctx.ingest([s])
        mine = _lib.talp_gpu_region_metrics(ctx.ctx, s.trace_id, _lib.TALP_GPU_ALL_REGIONS, stream, n_regions=R,
                                            check=False)[1]
        ctx.reset(s.trace_id)
    else:
        mine = []
        for r in range(R):
            m = _lib.talp_gpu_metrics()
            m.trace_id, m.region = s.trace_id, r
            mine.append(m)
    parts = exchange(mine, group)
    return [_lib.metrics_to_dict(_lib.talp_gpu_metrics_combine(ctx.ctx, parts[r], stream, check=False)[1])
            for r in range(R)]


def sharded_thread_metrics(ctx, t, proc_off, group=None, stream=None) -> list:
    """Host tree with threads of every region of trace `t` (host units =
    threads, grouped by proc_off) reduced across the ranks of the process
    group: this process ingests its block of whole processes into `ctx`,
    exchanges the thread-tree records and combines them."""
    import torch.distributed as dist
    world, me = dist.get_world_size(group), dist.get_rank(group)
    po = np.asarray(proc_off, np.int64)
    hoff = np.asarray(t.host_off, np.int64)
    doff = np.asarray(t.dev_off, np.int64)
    dstart = np.concatenate([[0], np.cumsum(np.asarray(t.devices_per_rank, np.int64))])
    rec = np.diff(hoff) + (doff[dstart[1:]] - doff[dstart[:-1]])
    procs = partition_processes(rec, po, world)[me]
    s = shard_of(t, units_of(po, procs))
    R = s.n_regions
    if procs.size:
        ctx.ingest([s])
        mine = _lib.talp_gpu_thread_metrics(ctx.ctx, s.trace_id, _lib.TALP_GPU_ALL_REGIONS,
                                            po[procs[0]:procs[-1] + 2] - po[procs[0]], stream, n_regions=R,
                                            check=False)[1]
        ctx.reset(s.trace_id)
    else:
        mine = [{f: 0 for f, _ in _lib.talp_gpu_thread_tree._fields_} for _ in range(R)]
        for r in range(R):
            mine[r].update(trace_id=s.trace_id, region=r)
    parts = exchange(mine, group, threads=True)
    out = []
    for r in range(R):
        live = [p for p in parts[r] if p["n_threads"]]
        out.append(_lib.talp_gpu_thread_metrics_combine(ctx.ctx, live, stream, check=False)[1])
    return out
