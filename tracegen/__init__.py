"""Seeded synthetic trace generator.

This module only produces inputs: per-rank host-state intervals and
per-device activity records, in the record layout the library ingests.  It
holds none of the efficiency arithmetic (no clipping, no unions, no ratios),
so both the CUDA path and the CPU oracle can be fed from it without sharing
any of the method.

Record layout (one trace):
  host_se    int64[N_host, 2]   {start_ns, end_ns}, CSR by rank (host_off)
  host_state uint8[N_host]      0 = useful, 1 = device offloading, 2 = MPI
  dev_se     int64[N_dev, 2]    {start_ns, end_ns}, CSR by (rank, device)
  dev_tag    uint8[N_dev]       kind << 5 | stream; kind 0 = kernel,
                                1 = H2D, 2 = D2H, 3 = D2D, 4 = memset
  region_window int64[R, n, 2]  per region and rank: [begin, end)

Every random draw comes from a Philox counter-based stream keyed by
(seed, trace, segment), so any single segment can be regenerated on its own
(this is how the full-size parity tests sample segments for the oracle).

Duration laws (all in integer nanoseconds):
  host    : state i.i.d. uniform over {useful, offload, MPI}; exponential
            durations with means 50 us / 5 us / 10 us; intervals back to back
            from t = 0, padded at the end with one offload interval (the host
            blocked on the device) up to the rank window end T_i.
  kernels : lognormal(mu = ln 20 us, sigma = 1) or bimodal 1 us / 500 us
            (80/20), times the rank work factor; each kernel stream is a
            sequential lane with exponential gaps sized for a target lane
            occupancy.
  copies  : lognormal(mu = ln 8 us, sigma = 0.7), H2D/D2H 50/50; 30% start
            uniformly inside a random kernel, the rest inside the gap after a
            random kernel.
Device records of one device are emitted sorted by start (merged over its
streams); `interleave_lanes` / `shuffle_segments` produce unsorted variants.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from concurrent.futures import ThreadPoolExecutor
import os

import numpy as np

KIND_KERNEL, KIND_H2D, KIND_D2H, KIND_D2D, KIND_MEMSET = 0, 1, 2, 3, 4
STATE_USEFUL, STATE_OFFLOAD, STATE_MPI = 0, 1, 2

US = 1000  # ns per microsecond


def make_tag(kind, stream):
    return ((np.asarray(kind, dtype=np.uint8) << 5) | (np.asarray(stream, dtype=np.uint8) & 31)).astype(np.uint8)


@dataclass
class Trace:
    trace_id: int
    n_ranks: int
    devices_per_rank: np.ndarray      # uint32[n]
    region_window: np.ndarray         # int64[R, n, 2]
    host_se: np.ndarray               # int64[Nh, 2]
    host_state: np.ndarray            # uint8[Nh]
    host_off: np.ndarray              # uint64[n + 1]
    dev_se: np.ndarray                # int64[Nd, 2]
    dev_tag: np.ndarray               # uint8[Nd]
    dev_off: np.ndarray               # uint64[m + 1]
    sorted_by_start: bool = True
    meta: dict = field(default_factory=dict)

    @property
    def n_regions(self) -> int:
        return int(self.region_window.shape[0])

    @property
    def m_devices(self) -> int:
        return int(self.dev_off.shape[0] - 1)

    @property
    def n_host(self) -> int:
        return int(self.host_se.shape[0])

    @property
    def n_dev(self) -> int:
        return int(self.dev_se.shape[0])

    @property
    def n_records(self) -> int:
        return self.n_host + self.n_dev

    @property
    def nbytes(self) -> int:
        """Algorithmic input bytes: 16 B {start,end} + 1 B tag/state per record."""
        return 17 * self.n_records

    def device_rank(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_ranks, dtype=np.int64), self.devices_per_rank.astype(np.int64))

    def dev_segment(self, g):
        a, b = int(self.dev_off[g]), int(self.dev_off[g + 1])
        return self.dev_se[a:b], self.dev_tag[a:b]

    def host_segment(self, i):
        a, b = int(self.host_off[i]), int(self.host_off[i + 1])
        return self.host_se[a:b], self.host_state[a:b]


# ----------------------------------------------------------------------------
# random streams


def _rng(seed: int, trace_id: int, domain: int, index: int) -> np.random.Generator:
    """Independent Philox-4x32-10 stream per (seed, trace, domain, index)."""
    k0 = (int(seed) & 0xFFFFFFFF) | ((int(trace_id) & 0xFFFFFFFF) << 32)
    k1 = ((int(domain) & 0xFF) << 56) | (int(index) & ((1 << 56) - 1))
    return np.random.Generator(np.random.Philox(key=np.array([k0, k1], dtype=np.uint64)))


D_HOST, D_DEV, D_TRACE, D_SHAPE, D_THREAD = 1, 2, 3, 4, 5


def _rint_pos(x):
    return np.maximum(np.rint(x), 1).astype(np.int64)


# ----------------------------------------------------------------------------
# segment laws


@dataclass
class DeviceLaw:
    kernel_law: str = "lognormal"        # or "bimodal"
    kernel_streams: tuple = (0,)
    copy_streams: tuple = (0,)
    occupancy: float = 0.7               # target kernel occupancy summed over lanes
    kernel_frac: float = 0.7
    copy_inside_frac: float = 0.3


def _kernel_durations(rng, n, law, work):
    if law == "lognormal":
        d = np.exp(rng.normal(math.log(20 * US), 1.0, n))
        mean = 20 * US * math.exp(0.5)
    elif law == "bimodal":
        d = np.where(rng.random(n) < 0.8, 1 * US, 500 * US).astype(np.float64)
        mean = 0.8 * US + 0.2 * 500 * US
    else:
        raise ValueError(law)
    return _rint_pos(d * work), mean * work


def device_segment(rng, n_events, law: DeviceLaw, work=1.0, t0=0):
    """One device's records, sorted by start; returns (se[n,2], tag[n])."""
    if n_events <= 0:
        return np.zeros((0, 2), np.int64), np.zeros(0, np.uint8)
    n_k = max(1, int(round(law.kernel_frac * n_events)))
    n_c = n_events - n_k
    kd, mean_k = _kernel_durations(rng, n_k, law.kernel_law, work)
    L = len(law.kernel_streams)
    rho_lane = min(law.occupancy / L, 0.95)
    mean_gap = mean_k * (1.0 - rho_lane) / rho_lane
    gaps = np.rint(rng.exponential(mean_gap, n_k)).astype(np.int64)
    ks = np.empty(n_k, np.int64)
    gap_next = np.empty(n_k, np.int64)
    kstream = np.empty(n_k, np.uint8)
    for lane in range(L):
        idx = np.arange(lane, n_k, L)
        if idx.size == 0:
            continue
        g = gaps[idx]
        d = kd[idx]
        start = t0 + np.cumsum(g + d) - d
        ks[idx] = start
        nxt = np.empty(idx.size, np.int64)
        nxt[:-1] = g[1:]
        nxt[-1] = int(round(mean_gap))
        gap_next[idx] = nxt
        kstream[idx] = law.kernel_streams[lane]
    ke = ks + kd
    if n_c > 0:
        which = rng.integers(0, n_k, n_c)
        inside = rng.random(n_c) < law.copy_inside_frac
        u = rng.random(n_c)
        cs = np.where(inside,
                      ks[which] + np.floor(u * kd[which]).astype(np.int64),
                      ke[which] + np.floor(u * gap_next[which]).astype(np.int64))
        cd = _rint_pos(np.exp(rng.normal(math.log(8 * US), 0.7, n_c)))
        ckind = np.where(rng.random(n_c) < 0.5, KIND_H2D, KIND_D2H).astype(np.uint8)
        cstream = np.asarray(law.copy_streams, np.uint8)[np.arange(n_c) % len(law.copy_streams)]
        starts = np.concatenate([ks, cs])
        ends = np.concatenate([ke, cs + cd])
        tags = np.concatenate([make_tag(np.zeros(n_k, np.uint8), kstream), make_tag(ckind, cstream)])
    else:
        starts, ends, tags = ks, ke, make_tag(np.zeros(n_k, np.uint8), kstream)
    order = np.argsort(starts, kind="stable")
    se = np.empty((n_events, 2), np.int64)
    se[:, 0] = starts[order]
    se[:, 1] = ends[order]
    return se, tags[order]


HOST_MEANS_NS = {STATE_USEFUL: 50 * US, STATE_OFFLOAD: 5 * US, STATE_MPI: 10 * US}


def host_segment(rng, n_events, t0=0):
    """Back-to-back host intervals from t0; returns (se[n,2], state[n])."""
    if n_events <= 0:
        return np.zeros((0, 2), np.int64), np.zeros(0, np.uint8)
    state = rng.integers(0, 3, n_events).astype(np.uint8)
    means = np.array([HOST_MEANS_NS[0], HOST_MEANS_NS[1], HOST_MEANS_NS[2]], np.float64)[state]
    dur = np.rint(rng.exponential(1.0, n_events) * means).astype(np.int64)
    ends = t0 + np.cumsum(dur)
    se = np.empty((n_events, 2), np.int64)
    se[:, 0] = ends - dur
    se[:, 1] = ends
    return se, state


def nested_regions(T, n_regions):
    """Region 0 = [0, T_i) per rank; region k = [k L/(2R), L - k L/(2R)), L = min T."""
    T = np.asarray(T, np.int64)
    n = T.shape[0]
    win = np.zeros((n_regions, n, 2), np.int64)
    win[0, :, 0] = 0
    win[0, :, 1] = T
    L = int(T.min()) if n else 0
    for k in range(1, n_regions):
        win[k, :, 0] = k * L // (2 * n_regions)
        win[k, :, 1] = L - k * L // (2 * n_regions)
    return win


# ----------------------------------------------------------------------------
# whole traces


def _pool_map(fn, items, threads):
    if threads <= 1 or len(items) <= 1:
        return [fn(x) for x in items]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(fn, items))


def build_trace(seed, trace_id, devices_per_rank, dev_events, host_events, law: DeviceLaw,
                work=None, n_regions=1, threads=None, pad_state=STATE_OFFLOAD):
    """Assemble one trace from per-device and per-rank event counts.

    dev_events: int array [m] (device events per device, rank-major order)
    host_events: int array [n]
    work: float array [n] (rank work factor multiplying kernel durations)
    """
    dpr = np.asarray(devices_per_rank, np.uint32)
    n = dpr.shape[0]
    m = int(dpr.sum())
    dev_events = np.asarray(dev_events, np.int64).reshape(m)
    host_events = np.asarray(host_events, np.int64).reshape(n)
    if work is None:
        work = np.ones(n)
    dev_rank = np.repeat(np.arange(n), dpr.astype(np.int64))
    if threads is None:
        threads = min(32, os.cpu_count() or 1)

    def dev_job(g):
        rng = _rng(seed, trace_id, D_DEV, g)
        return device_segment(rng, int(dev_events[g]), law, float(work[dev_rank[g]]))

    def host_job(i):
        rng = _rng(seed, trace_id, D_HOST, i)
        return host_segment(rng, int(host_events[i]))

    devs = _pool_map(dev_job, list(range(m)), threads)
    hosts = _pool_map(host_job, list(range(n)), threads)

    dev_off = np.zeros(m + 1, np.uint64)
    dev_off[1:] = np.cumsum([d[0].shape[0] for d in devs])
    dev_se = np.concatenate([d[0] for d in devs]) if m else np.zeros((0, 2), np.int64)
    dev_tag = np.concatenate([d[1] for d in devs]) if m else np.zeros(0, np.uint8)
    del devs

    # rank window end: the later of the host timeline end and its devices' last end
    T = np.zeros(n, np.int64)
    g = 0
    for i in range(n):
        t = int(hosts[i][0][-1, 1]) if hosts[i][0].shape[0] else 0
        for _ in range(int(dpr[i])):
            a, b = int(dev_off[g]), int(dev_off[g + 1])
            if b > a:
                t = max(t, int(dev_se[a:b, 1].max()))
            g += 1
        T[i] = max(t, 1)
    host_parts, state_parts = [], []
    host_off = np.zeros(n + 1, np.uint64)
    for i in range(n):
        se, st = hosts[i]
        end = int(se[-1, 1]) if se.shape[0] else 0
        if T[i] > end:
            se = np.concatenate([se, np.array([[end, T[i]]], np.int64)])
            st = np.concatenate([st, np.array([pad_state], np.uint8)])
        host_parts.append(se)
        state_parts.append(st)
        host_off[i + 1] = host_off[i] + se.shape[0]
    host_se = np.concatenate(host_parts) if n else np.zeros((0, 2), np.int64)
    host_state = np.concatenate(state_parts) if n else np.zeros(0, np.uint8)
    return Trace(trace_id=trace_id, n_ranks=n, devices_per_rank=dpr,
                 region_window=nested_regions(T, n_regions),
                 host_se=np.ascontiguousarray(host_se), host_state=host_state, host_off=host_off,
                 dev_se=np.ascontiguousarray(dev_se), dev_tag=dev_tag, dev_off=dev_off,
                 sorted_by_start=True)


# ----------------------------------------------------------------------------
# the five workloads (with a size scale for parity tests)


def single_trace_small(seed=0x7A1F, scale=1.0, trace_id=0):
    """4 ranks x 1 GPU x 1 stream; 10k host + 10k device events per rank; 1 region."""
    n = 4
    ev = max(1, int(round(10_000 * scale)))
    law = DeviceLaw("lognormal", (0,), (0,), occupancy=0.7)
    t = build_trace(seed, trace_id, [1] * n, [ev] * n, [ev] * n, law, n_regions=1)
    t.meta.update(workload="single trace, 4 ranks x 1 GPU x 1 stream", scale=scale)
    return t


def plain_large(seed=0x7A1F + 1, scale=1.0, trace_id=1, n_ranks=64, gpus_per_rank=4, threads=None):
    """64 ranks x 4 GPUs x 4 streams; 2M device events/GPU, 1M host/rank; 4 nested regions."""
    dev_ev = max(1, int(round(2_000_000 * scale)))
    host_ev = max(1, int(round(1_000_000 * scale)))
    m = n_ranks * gpus_per_rank
    work = 0.7 + 0.3 * _rng(seed, trace_id, D_SHAPE, 0).random(n_ranks)
    law = DeviceLaw("lognormal", (0, 1, 2, 3), (2, 3), occupancy=0.7)
    t = build_trace(seed, trace_id, [gpus_per_rank] * n_ranks, [dev_ev] * m, [host_ev] * n_ranks,
                    law, work=work, n_regions=4, threads=threads)
    t.meta.update(workload=f"plain large single trace, {n_ranks} ranks x {gpus_per_rank} GPUs x 4 streams",
                  scale=scale)
    return t


def scale_trace(seed=0x7A1F + 3, scale=1.0, trace_id=3, n_ranks=1024, gpus_per_rank=4, threads=None):
    """1024 ranks x 4 GPUs x 8 streams, bimodal kernels, 20% of ranks with 1.5x events."""
    base = max(1, int(round(222_000 * scale)))
    host_ev = max(1, int(round(100_000 * scale)))
    rng = _rng(seed, trace_id, D_SHAPE, 0)
    heavy = np.zeros(n_ranks, bool)
    heavy[rng.permutation(n_ranks)[: int(round(0.2 * n_ranks))]] = True
    per_rank = np.where(heavy, int(round(1.5 * base)), base)
    dev_ev = np.repeat(per_rank, gpus_per_rank)
    law = DeviceLaw("bimodal", tuple(range(8)), (6, 7), occupancy=0.7)
    t = build_trace(seed, trace_id, [gpus_per_rank] * n_ranks, dev_ev, [host_ev] * n_ranks, law,
                    n_regions=4, threads=threads)
    t.meta.update(workload=f"scale trace, {n_ranks} ranks x {gpus_per_rank} GPUs x 8 streams", scale=scale)
    return t


def batched_shapes(seed=0x7A1F + 2, n_traces=4096, max_ranks=512, max_gpus=8,
                   ev_lo=1_000, ev_hi=1_000_000):
    """Per-trace shapes of the batched workload: ranks log-uniform in [1, max_ranks],
    GPUs per rank uniform in [1, max_gpus], events per GPU log-uniform in [ev_lo, ev_hi]
    (host intervals per rank = device events per GPU)."""
    rng = _rng(seed, 0, D_SHAPE, 1)
    ranks = np.clip(np.floor(np.exp(rng.uniform(0, math.log(max_ranks + 1), n_traces))), 1, max_ranks).astype(np.int64)
    gpus = rng.integers(1, max_gpus + 1, n_traces)
    ev = np.clip(np.rint(np.exp(rng.uniform(math.log(ev_lo), math.log(ev_hi), n_traces))), ev_lo, ev_hi).astype(np.int64)
    return ranks, gpus, ev


def batched_trace(k, ranks, gpus, ev, seed=0x7A1F + 2, n_regions=8, threads=1):
    n = int(ranks[k])
    g = int(gpus[k])
    e = int(ev[k])
    law = DeviceLaw("lognormal", (0,), (0,), occupancy=0.7)
    work = 0.7 + 0.3 * _rng(seed, k, D_SHAPE, 2).random(n)
    t = build_trace(seed, k, [g] * n, [e] * (n * g), [e] * n, law, work=work,
                    n_regions=n_regions, threads=threads)
    t.meta.update(workload="batched member", index=k)
    return t


def batched_trace_fast(k, ranks, gpus, ev, seed=0x7A1F + 2, n_regions=8, ev_scale=1.0):
    """One member of the batched workload, generated with whole-trace array
    operations (one Philox stream per trace, so a trace, not a segment, is
    the unit that can be regenerated alone).  Same laws as the small single
    trace: one kernel stream at occupancy 0.7 with lognormal kernels times
    the rank work factor, 30% copies (30% inside a kernel), back-to-back host
    intervals padded with one offload interval to the rank window end."""
    n = int(ranks[k])
    g = int(gpus[k])
    E = max(1, int(round(int(ev[k]) * ev_scale)))
    m = n * g
    rng = _rng(seed, k, D_TRACE, 3)
    work = 0.7 + 0.3 * _rng(seed, k, D_SHAPE, 2).random(n)
    wdev = np.repeat(work, g)[:, None]
    n_k = max(1, int(round(0.7 * E)))
    n_c = E - n_k
    kd = np.maximum(np.rint(np.exp(rng.normal(math.log(20 * US), 1.0, (m, n_k))) * wdev), 1).astype(np.int64)
    mean_k = 20 * US * math.exp(0.5) * wdev
    gaps = np.rint(rng.exponential(1.0, (m, n_k)) * (mean_k * (1 - 0.7) / 0.7)).astype(np.int64)
    ks = np.cumsum(gaps + kd, axis=1) - kd
    ke = ks + kd
    gap_next = np.empty_like(gaps)
    gap_next[:, :-1] = gaps[:, 1:]
    gap_next[:, -1] = np.rint(mean_k[:, 0] * (1 - 0.7) / 0.7).astype(np.int64)
    if n_c > 0:
        which = rng.integers(0, n_k, (m, n_c))
        inside = rng.random((m, n_c)) < 0.3
        u = rng.random((m, n_c))
        rows = np.arange(m)[:, None]
        cs = np.where(inside, ks[rows, which] + np.floor(u * kd[rows, which]).astype(np.int64),
                      ke[rows, which] + np.floor(u * gap_next[rows, which]).astype(np.int64))
        cd = np.maximum(np.rint(np.exp(rng.normal(math.log(8 * US), 0.7, (m, n_c)))), 1).astype(np.int64)
        ckind = np.where(rng.random((m, n_c)) < 0.5, KIND_H2D, KIND_D2H).astype(np.uint8)
        starts = np.concatenate([ks, cs], axis=1)
        ends = np.concatenate([ke, cs + cd], axis=1)
        tags = np.concatenate([np.zeros((m, n_k), np.uint8), (ckind << 5)], axis=1)
    else:
        starts, ends, tags = ks, ke, np.zeros((m, n_k), np.uint8)
    order = np.argsort(starts, axis=1, kind="stable")
    starts = np.take_along_axis(starts, order, 1)
    ends = np.take_along_axis(ends, order, 1)
    tags = np.take_along_axis(tags, order, 1)
    dev_se = np.empty((m * E, 2), np.int64)
    dev_se[:, 0] = starts.reshape(-1)
    dev_se[:, 1] = ends.reshape(-1)
    dev_end = ends.max(axis=1).reshape(n, g).max(axis=1)
    # host: E intervals per rank + one padding interval
    state = rng.integers(0, 3, (n, E)).astype(np.uint8)
    means = np.array([HOST_MEANS_NS[0], HOST_MEANS_NS[1], HOST_MEANS_NS[2]], np.float64)[state]
    dur = np.rint(rng.exponential(1.0, (n, E)) * means).astype(np.int64)
    hend = np.cumsum(dur, axis=1)
    T = np.maximum(np.maximum(hend[:, -1], dev_end), 1)
    hs = np.empty((n, E + 1), np.int64)
    he = np.empty((n, E + 1), np.int64)
    hs[:, :E] = hend - dur
    he[:, :E] = hend
    hs[:, E] = hend[:, -1]
    he[:, E] = T
    hst = np.empty((n, E + 1), np.uint8)
    hst[:, :E] = state
    hst[:, E] = STATE_OFFLOAD
    host_se = np.empty((n * (E + 1), 2), np.int64)
    host_se[:, 0] = hs.reshape(-1)
    host_se[:, 1] = he.reshape(-1)
    return Trace(trace_id=k, n_ranks=n, devices_per_rank=np.full(n, g, np.uint32),
                 region_window=nested_regions(T, n_regions), host_se=host_se, host_state=hst.reshape(-1),
                 host_off=(np.arange(n + 1, dtype=np.uint64) * np.uint64(E + 1)),
                 dev_se=dev_se, dev_tag=tags.reshape(-1).astype(np.uint8),
                 dev_off=(np.arange(m + 1, dtype=np.uint64) * np.uint64(E)),
                 sorted_by_start=True, meta=dict(workload="batched member", index=k, events_per_gpu=E))


def batched_workload(n_traces=4096, ev_lo=5, ev_hi=5000, seed=0x7A1F + 2, n_regions=8, threads=None):
    """The batched workload: n_traces traces with ranks log-uniform in
    [1, 512], GPUs per rank uniform in [1, 8], events per GPU (= host
    intervals per rank) log-uniform in [ev_lo, ev_hi]."""
    ranks, gpus, ev = batched_shapes(seed=seed, n_traces=n_traces, ev_lo=ev_lo, ev_hi=ev_hi)
    if threads is None:
        threads = min(32, os.cpu_count() or 1)
    return _pool_map(lambda k: batched_trace_fast(k, ranks, gpus, ev, seed=seed, n_regions=n_regions),
                     list(range(n_traces)), threads)


# ----------------------------------------------------------------------------
# small adversarial traces for exact checks


def rescale_time(t: Trace, scale: int, offset: int = 0) -> Trace:
    """The same trace with every timestamp (records and windows) mapped to
    t * scale + offset: spans of 2^32 ns and more, or values near 2^62."""
    def f(a):
        return (a.astype(np.int64) * np.int64(scale) + np.int64(offset)).astype(np.int64)
    return Trace(trace_id=t.trace_id, n_ranks=t.n_ranks, devices_per_rank=t.devices_per_rank,
                 region_window=f(t.region_window), host_se=f(t.host_se), host_state=t.host_state,
                 host_off=t.host_off, dev_se=f(t.dev_se), dev_tag=t.dev_tag, dev_off=t.dev_off,
                 sorted_by_start=t.sorted_by_start, meta=dict(t.meta, scale=scale, offset=offset))


def tiny_trace(seed, trace_id=0, max_ranks=3, max_devs=2, max_events=64, horizon=4096,
               n_regions=None, tiled_host=None, allow_empty=True, kinds=(0, 1, 2, 3, 4), streams=4):
    """Random small trace: arbitrary overlaps, zero-length intervals, empty
    segments, touching intervals, windows that straddle / miss the data."""
    rng = _rng(seed, trace_id, D_TRACE, 7)
    n = int(rng.integers(1, max_ranks + 1))
    dpr = rng.integers(0 if allow_empty else 1, max_devs + 1, n).astype(np.uint32)
    if dpr.sum() == 0:
        dpr[0] = 1
    m = int(dpr.sum())
    R = int(n_regions if n_regions is not None else rng.integers(1, 4))
    if tiled_host is None:
        tiled_host = bool(rng.random() < 0.7)
    # device records
    segs, tags = [], []
    for g in range(m):
        k = int(rng.integers(0 if allow_empty else 1, max_events + 1))
        s = rng.integers(0, horizon, k)
        mode = rng.random()
        if mode < 0.15:
            d = rng.integers(1, 64, k)                     # zero-length heavy
            d[rng.random(k) < 0.5] = 0
        elif mode < 0.3:
            d = rng.integers(0, horizon // 2, k)           # long, nested
        else:
            d = rng.integers(0, 200, k)
        e = np.minimum(s + d, horizon + 512)
        order = np.argsort(s, kind="stable")
        se = np.stack([s[order], e[order]], axis=1).astype(np.int64)
        kind = rng.choice(np.asarray(kinds, np.uint8), k)
        st = rng.integers(0, streams, k).astype(np.uint8)
        segs.append(se)
        tags.append(make_tag(kind, st))
    dev_off = np.zeros(m + 1, np.uint64)
    dev_off[1:] = np.cumsum([x.shape[0] for x in segs])
    dev_se = np.concatenate(segs) if m else np.zeros((0, 2), np.int64)
    dev_tag = np.concatenate(tags) if m else np.zeros(0, np.uint8)
    # host records
    hparts, sparts = [], []
    host_off = np.zeros(n + 1, np.uint64)
    T = np.zeros(n, np.int64)
    for i in range(n):
        k = int(rng.integers(0 if allow_empty else 1, max_events + 1))
        if tiled_host:
            d = rng.integers(0, 300, k)
            e = np.cumsum(d)
            se = np.stack([e - d, e], axis=1).astype(np.int64)
        else:
            s = rng.integers(0, horizon, k)
            d = rng.integers(0, 300, k)
            se = np.stack([s, s + d], axis=1).astype(np.int64)
        hparts.append(se)
        sparts.append(rng.integers(0, 3, k).astype(np.uint8))
        host_off[i + 1] = host_off[i] + k
        T[i] = int(se[:, 1].max()) if k else 0
    host_se = np.concatenate(hparts) if n else np.zeros((0, 2), np.int64)
    host_state = np.concatenate(sparts) if n else np.zeros(0, np.uint8)
    # windows
    win = np.zeros((R, n, 2), np.int64)
    for r in range(R):
        for i in range(n):
            mode = rng.random()
            if tiled_host and r == 0:
                a, b = 0, int(T[i])
            elif mode < 0.1:
                a = b = int(rng.integers(0, horizon))      # empty window
            elif mode < 0.2:
                a, b = horizon + 1000, horizon + 2000      # misses everything
            else:
                a = int(rng.integers(-100, horizon))
                b = int(rng.integers(a, horizon + 600))
            win[r, i] = (a, b)
    return Trace(trace_id=trace_id, n_ranks=n, devices_per_rank=dpr, region_window=win,
                 host_se=host_se, host_state=host_state, host_off=host_off,
                 dev_se=dev_se, dev_tag=dev_tag, dev_off=dev_off, sorted_by_start=True,
                 meta=dict(workload="tiny", tiled_host=tiled_host))


def random_trace(seed, trace_id=0, n_ranks=3, devices_per_rank=2, dev_events=5000, host_events=3000,
                 n_regions=3, law=None):
    """A mid-size trace from the physical laws with explicit sizes (parity tests)."""
    if law is None:
        law = DeviceLaw("lognormal", (0, 1, 2), (1, 2), occupancy=0.8)
    dpr = [devices_per_rank] * n_ranks if np.isscalar(devices_per_rank) else list(devices_per_rank)
    m = int(sum(dpr))
    dev_ev = [dev_events] * m if np.isscalar(dev_events) else list(dev_events)
    host_ev = [host_events] * n_ranks if np.isscalar(host_events) else list(host_events)
    work = 0.7 + 0.3 * _rng(seed, trace_id, D_SHAPE, 3).random(n_ranks)
    return build_trace(seed, trace_id, dpr, dev_ev, host_ev, law, work=work, n_regions=n_regions, threads=1)


# ----------------------------------------------------------------------------
# threads: one host unit per thread, grouped into processes


def worker_segment(rng, master_se, master_state, busy_frac):
    """Fork-join worker of a process: inside each useful interval of its master
    it is busy from the interval start for busy_frac x U(0.8, 1) of the
    interval (useful; 10% of them device offloading, 2% MPI), idle elsewhere."""
    mask = master_state == STATE_USEFUL
    se = master_se[mask]
    k = se.shape[0]
    d = np.floor((se[:, 1] - se[:, 0]) * busy_frac * rng.uniform(0.8, 1.0, k)).astype(np.int64)
    u = rng.random(k)
    state = np.where(u < 0.02, STATE_MPI, np.where(u < 0.12, STATE_OFFLOAD, STATE_USEFUL)).astype(np.uint8)
    keep = d > 0
    out = np.empty((int(keep.sum()), 2), np.int64)
    out[:, 0] = se[keep, 0]
    out[:, 1] = se[keep, 0] + d[keep]
    return out, state[keep]


def add_threads(trace: Trace, threads, seed=0x7A1F + 5, imbalance=0.3, pool=None) -> Trace:
    """Expand each rank of `trace` into a process of T_i threads: unit 0 of the
    process is the rank itself (its master thread, owning its devices), the
    other T_i - 1 units are fork-join workers (worker_segment) with busy
    fraction 1 - imbalance x U(0, 1) each.  Every unit keeps its process's
    region windows.  meta["proc_off"] = uint32[n + 1] groups the units."""
    n = int(trace.n_ranks)
    T = np.full(n, int(threads), np.int64) if np.isscalar(threads) else np.asarray(threads, np.int64)
    assert T.shape == (n,) and np.all(T >= 1)
    proc_off = np.zeros(n + 1, np.uint32)
    proc_off[1:] = np.cumsum(T)
    nT = int(proc_off[-1])

    def proc_job(i):
        mse, mst = trace.host_segment(i)
        rng = _rng(seed, trace.trace_id, D_THREAD, i)
        fr = 1.0 - imbalance * rng.random(int(T[i]) - 1)
        parts = [(mse, mst)]
        for w in range(int(T[i]) - 1):
            parts.append(worker_segment(_rng(seed, trace.trace_id, D_THREAD, (i << 16) + w + 1), mse, mst, fr[w]))
        return parts

    if pool is None:
        pool = min(32, os.cpu_count() or 1)
    units = [u for parts in _pool_map(proc_job, list(range(n)), pool) for u in parts]
    host_off = np.zeros(nT + 1, np.uint64)
    host_off[1:] = np.cumsum([u[0].shape[0] for u in units])
    dpr = np.zeros(nT, np.uint32)
    dpr[proc_off[:-1]] = trace.devices_per_rank
    win = np.repeat(trace.region_window, T, axis=1)
    return Trace(trace_id=trace.trace_id, n_ranks=nT, devices_per_rank=dpr, region_window=np.ascontiguousarray(win),
                 host_se=np.ascontiguousarray(np.concatenate([u[0] for u in units])),
                 host_state=np.concatenate([u[1] for u in units]), host_off=host_off,
                 dev_se=trace.dev_se, dev_tag=trace.dev_tag, dev_off=trace.dev_off,
                 sorted_by_start=trace.sorted_by_start,
                 meta={**trace.meta, "proc_off": proc_off, "threads": T})


def threaded_large(seed=0x7A1F + 1, scale=1.0, trace_id=1, threads=8, pool=None):
    """The plain large trace with 8 threads per rank: 64 processes x 8 threads
    (one master + 7 fork-join workers) x 4 GPUs; 4 nested regions."""
    t = add_threads(plain_large(seed, scale, trace_id, threads=pool), threads, pool=pool)
    t.meta.update(workload=f"plain large single trace with {threads} threads per rank, 64 ranks x 4 GPUs x 4 streams")
    return t


# ----------------------------------------------------------------------------
# unsorted variants (ingest must sort these)


def interleave_lanes(trace: Trace) -> Trace:
    """Per device, regroup records stream by stream (each stream still in start
    order): the order a per-stream activity buffer would deliver them."""
    se = trace.dev_se.copy()
    tag = trace.dev_tag.copy()
    for g in range(trace.m_devices):
        a, b = int(trace.dev_off[g]), int(trace.dev_off[g + 1])
        if b - a < 2:
            continue
        order = np.argsort(tag[a:b] & 31, kind="stable")
        se[a:b] = se[a:b][order]
        tag[a:b] = tag[a:b][order]
    return _with_dev(trace, se, tag)


def shuffle_segments(trace: Trace, seed=1, frac=1.0) -> Trace:
    """Randomly permute the records of a fraction of the device segments."""
    rng = _rng(seed, trace.trace_id, D_TRACE, 11)
    se = trace.dev_se.copy()
    tag = trace.dev_tag.copy()
    for g in range(trace.m_devices):
        a, b = int(trace.dev_off[g]), int(trace.dev_off[g + 1])
        if b - a < 2 or rng.random() >= frac:
            continue
        p = rng.permutation(b - a)
        se[a:b] = se[a:b][p]
        tag[a:b] = tag[a:b][p]
    return _with_dev(trace, se, tag)


def split_runs(trace: Trace, k: int, seed=3) -> Trace:
    """Deal each device's records (in start order) into k groups at random
    and lay the groups end to end: every segment becomes at most k sorted
    runs, as records grouped by stream are."""
    rng = _rng(seed, trace.trace_id, D_TRACE, 31)
    se = trace.dev_se.copy()
    tag = trace.dev_tag.copy()
    for g in range(trace.m_devices):
        a, b = int(trace.dev_off[g]), int(trace.dev_off[g + 1])
        if b - a < 2:
            continue
        grp = rng.integers(0, k, b - a)
        order = np.argsort(grp, kind="stable")
        se[a:b] = se[a:b][order]
        tag[a:b] = tag[a:b][order]
    return _with_dev(trace, se, tag)


@dataclass
class RawTrace:
    """A trace's device records as an activity API delivers them: per rank,
    one buffer of all its devices' records with the device index within
    the rank, the streams interleaved in completion order (a record is
    delivered when it and every earlier record of its stream are done)."""
    trace: Trace
    raw_se: np.ndarray       # int64[N, 2]
    raw_tag: np.ndarray      # uint8[N]
    raw_dev: np.ndarray      # uint8[N]
    raw_off: np.ndarray      # uint64[n + 1]
    stream_mask: np.ndarray = None   # uint32[n, 8]: declared streams of each device (hold-back)


def stream_masks(trace: Trace) -> np.ndarray:
    """uint32[n, 8]: bit s of [i, d] set when device d of rank i has a
    record on stream s."""
    dpr = np.asarray(trace.devices_per_rank, np.int64)
    cnt = np.diff(trace.dev_off.astype(np.int64))
    g = np.repeat(np.arange(int(dpr.sum())), cnt)
    rank = np.repeat(np.repeat(np.arange(trace.n_ranks), dpr), cnt)
    local = g - np.concatenate([[0], np.cumsum(dpr)])[rank]
    out = np.zeros((trace.n_ranks, 8), np.uint32)
    np.bitwise_or.at(out, (rank, local), np.left_shift(np.uint32(1), (trace.dev_tag & 31).astype(np.uint32)))
    return out


def raw_deliveries(raw: RawTrace, n_calls: int, seed=7) -> list:
    """Cut every rank's delivery sequence at random into n_calls consecutive
    buffers; part j holds buffer j of every rank (a RawTrace whose trace
    has the whole trace's windows, the host records in part 0 only, and no
    device records of its own), with the trace's stream masks."""
    t = raw.trace
    rng = _rng(seed, t.trace_id, D_TRACE, 41)
    masks = stream_masks(t)
    off = raw.raw_off.astype(np.int64)
    cuts = np.zeros((t.n_ranks, n_calls + 1), np.int64)
    for i in range(t.n_ranks):
        c = np.sort(rng.integers(0, off[i + 1] - off[i] + 1, size=n_calls - 1))
        cuts[i] = np.concatenate([[0], c, [off[i + 1] - off[i]]])
    m = int(np.asarray(t.devices_per_rank, np.int64).sum())
    parts = []
    for j in range(n_calls):
        idx = np.concatenate([np.arange(off[i] + cuts[i, j], off[i] + cuts[i, j + 1]) for i in range(t.n_ranks)])
        roff = np.zeros(t.n_ranks + 1, np.uint64)
        roff[1:] = np.cumsum(cuts[:, j + 1] - cuts[:, j])
        if j == 0:
            hse, hst, hoff = t.host_se, t.host_state, t.host_off
        else:
            hse, hst, hoff = np.zeros((0, 2), np.int64), np.zeros(0, np.uint8), np.zeros(t.n_ranks + 1, np.uint64)
        pt = Trace(trace_id=t.trace_id, n_ranks=t.n_ranks, devices_per_rank=t.devices_per_rank,
                   region_window=t.region_window, host_se=hse, host_state=hst, host_off=hoff,
                   dev_se=np.zeros((0, 2), np.int64), dev_tag=np.zeros(0, np.uint8),
                   dev_off=np.zeros(m + 1, np.uint64), sorted_by_start=True, meta=dict(t.meta))
        parts.append(RawTrace(pt, np.ascontiguousarray(raw.raw_se[idx]), np.ascontiguousarray(raw.raw_tag[idx]),
                              np.ascontiguousarray(raw.raw_dev[idx]), roff, masks))
    return parts


def to_raw(trace: Trace) -> RawTrace:
    dpr = np.asarray(trace.devices_per_rank, np.int64)
    m = int(dpr.sum())
    cnt = np.diff(trace.dev_off.astype(np.int64))
    g = np.repeat(np.arange(m), cnt)                                  # global device of each record
    rank = np.repeat(np.repeat(np.arange(trace.n_ranks), dpr), cnt)
    local = g - np.concatenate([[0], np.cumsum(dpr)])[rank]
    lane = g * 32 + (trace.dev_tag & 31).astype(np.int64)
    # per (device, stream) lane in start order; delivery key: the running
    # maximum end along the lane (a record is done when it and all before it
    # in its stream are), computed for all lanes at once by lifting each
    # lane above the previous ones
    if trace.sorted_by_start:
        small = lane.astype(np.int16) if m * 32 < (1 << 15) else lane   # 16-bit keys sort by radix
        order = np.argsort(small, kind="stable")   # each device already in start order
    else:
        order = np.lexsort((trace.dev_se[:, 0], lane))
    se, tag, lane, rank, local = trace.dev_se[order], trace.dev_tag[order], lane[order], rank[order], local[order]
    if se.shape[0]:
        lo = int(se[:, 1].min())
        span = int(se[:, 1].max()) - lo + 1
        seg = np.concatenate([[0], np.cumsum(lane[1:] != lane[:-1])])
        key = np.maximum.accumulate((se[:, 1] - lo) + seg * span) - seg * span
    else:
        key = np.zeros(0, np.int64)
    d = np.argsort((rank.astype(np.int64) << 42) | key, kind="stable") if key.size and int(key.max()) < (1 << 42) \
        else np.lexsort((key, rank))
    off = np.zeros(trace.n_ranks + 1, np.uint64)
    off[1:] = np.cumsum(np.bincount(rank, minlength=trace.n_ranks))
    return RawTrace(trace, np.ascontiguousarray(se[d]), np.ascontiguousarray(tag[d]),
                    np.ascontiguousarray(local[d].astype(np.uint8)), off)


def _with_dev(trace, se, tag):
    return Trace(trace_id=trace.trace_id, n_ranks=trace.n_ranks, devices_per_rank=trace.devices_per_rank,
                 region_window=trace.region_window, host_se=trace.host_se, host_state=trace.host_state,
                 host_off=trace.host_off, dev_se=se, dev_tag=tag, dev_off=trace.dev_off,
                 sorted_by_start=False, meta=dict(trace.meta))


# ----------------------------------------------------------------------------
# streamed delivery: a trace cut into time slices (activity buffers handed
# over while the application runs)


@dataclass
class Slice:
    host_se: np.ndarray
    host_state: np.ndarray
    host_off: np.ndarray
    dev_se: np.ndarray
    dev_tag: np.ndarray
    dev_off: np.ndarray
    sorted_by_start: bool = True

    @property
    def n_records(self) -> int:
        return int(self.host_se.shape[0] + self.dev_se.shape[0])


def random_cuts(trace: Trace, n_slices: int, seed=5) -> np.ndarray:
    """n_slices - 1 increasing cut times drawn uniformly over the trace's span
    of start times."""
    starts = np.concatenate([trace.host_se[:, 0], trace.dev_se[:, 0]])
    if starts.size == 0 or n_slices < 2:
        return np.zeros(0, np.int64)
    lo, hi = int(starts.min()), int(starts.max()) + 1
    c = _rng(seed, trace.trace_id, D_TRACE, 21).integers(lo, hi, size=n_slices - 1)
    return np.sort(c).astype(np.int64)


def _keep(se, tag, off, mask):
    seg = np.repeat(np.arange(off.shape[0] - 1), np.diff(off.astype(np.int64)))
    counts = np.bincount(seg[mask], minlength=off.shape[0] - 1)
    new_off = np.zeros(off.shape[0], np.uint64)
    new_off[1:] = np.cumsum(counts)
    return np.ascontiguousarray(se[mask]), np.ascontiguousarray(tag[mask]), new_off


def time_slices(trace: Trace, cuts: np.ndarray, shuffle_seed=None) -> list:
    """Slice k holds, per rank and device, the records whose start lies in
    [cuts[k-1], cuts[k]) (open at both ends of the list), in the trace's own
    order.  With shuffle_seed, odd slices have their device segments
    permuted (the served form must sort them) and are flagged unsorted."""
    hk = np.searchsorted(cuts, trace.host_se[:, 0], side="right")
    dk = np.searchsorted(cuts, trace.dev_se[:, 0], side="right")
    out = []
    for k in range(cuts.shape[0] + 1):
        hse, hst, hoff = _keep(trace.host_se, trace.host_state, trace.host_off, hk == k)
        dse, dtg, doff = _keep(trace.dev_se, trace.dev_tag, trace.dev_off, dk == k)
        sl = Slice(hse, hst, hoff, dse, dtg, doff, sorted_by_start=trace.sorted_by_start)
        if shuffle_seed is not None and k % 2 == 1:
            rng = _rng(shuffle_seed, trace.trace_id, D_TRACE, 100 + k)
            for g in range(doff.shape[0] - 1):
                a, b = int(doff[g]), int(doff[g + 1])
                if b - a > 1:
                    p = rng.permutation(b - a)
                    dse[a:b] = dse[a:b][p]
                    dtg[a:b] = dtg[a:b][p]
            sl.sorted_by_start = False
        out.append(sl)
    return out


def prefix_trace(trace: Trace, cuts: np.ndarray, k: int) -> Trace:
    """The trace restricted to slices 0..k of time_slices(trace, cuts)."""
    hk = np.searchsorted(cuts, trace.host_se[:, 0], side="right")
    dk = np.searchsorted(cuts, trace.dev_se[:, 0], side="right")
    hse, hst, hoff = _keep(trace.host_se, trace.host_state, trace.host_off, hk <= k)
    dse, dtg, doff = _keep(trace.dev_se, trace.dev_tag, trace.dev_off, dk <= k)
    return Trace(trace_id=trace.trace_id, n_ranks=trace.n_ranks, devices_per_rank=trace.devices_per_rank,
                 region_window=trace.region_window, host_se=hse, host_state=hst, host_off=hoff, dev_se=dse,
                 dev_tag=dtg, dev_off=doff, sorted_by_start=trace.sorted_by_start, meta=dict(trace.meta))


@dataclass
class ServingJob:
    """One monitored job of the serving workload: a base trace cut into
    period batches by record count; batch q of the stream is base batch
    q mod P with every timestamp shifted by (q // P) * span."""
    job_id: int
    trace: Trace
    batches: list            # [Slice] * P
    span: int                # > every timestamp of the base trace
    n_regions: int

    def batch(self, q: int) -> Slice:
        b = self.batches[q % len(self.batches)]
        shift = np.int64((q // len(self.batches)) * self.span)
        if shift == 0:
            return b
        return Slice(b.host_se + shift, b.host_state, b.host_off, b.dev_se + shift, b.dev_tag, b.dev_off,
                     b.sorted_by_start)

    def windows(self, n_batches: int) -> np.ndarray:
        """Nested region windows over the time the first n_batches cover."""
        cycles = (max(1, n_batches) + len(self.batches) - 1) // len(self.batches)
        return nested_regions(np.full(self.trace.n_ranks, cycles * self.span, np.int64), self.n_regions)

    def prefix(self, n_batches: int, windows: np.ndarray) -> Trace:
        """The trace made of the first n_batches batches of the stream."""
        parts = [self.batch(q) for q in range(n_batches)]
        def cat(attr_se, attr_tag, attr_off, n_seg):
            if not parts:
                return np.zeros((0, 2), np.int64), np.zeros(0, np.uint8), np.zeros(n_seg + 1, np.uint64)
            se = np.concatenate([getattr(p, attr_se) for p in parts])
            tag = np.concatenate([getattr(p, attr_tag) for p in parts])
            seg = np.concatenate([np.repeat(np.arange(n_seg), np.diff(getattr(p, attr_off).astype(np.int64)))
                                  for p in parts])
            order = np.argsort(seg, kind="stable")
            off = np.zeros(n_seg + 1, np.uint64)
            off[1:] = np.cumsum(np.bincount(seg, minlength=n_seg))
            return se[order], tag[order], off
        t = self.trace
        hse, hst, hoff = cat("host_se", "host_state", "host_off", t.n_ranks)
        dse, dtg, doff = cat("dev_se", "dev_tag", "dev_off", t.m_devices)
        return Trace(trace_id=self.job_id, n_ranks=t.n_ranks, devices_per_rank=t.devices_per_rank,
                     region_window=windows, host_se=hse, host_state=hst, host_off=hoff, dev_se=dse, dev_tag=dtg,
                     dev_off=doff, sorted_by_start=True, meta=dict(workload="serving prefix", batches=n_batches))


def serving_jobs(n_jobs=256, seed=0x7A1F + 4, period=8, rank_lo=8, rank_hi=256, gpus_hi=4, batch_lo=1_000,
                 batch_hi=100_000, n_regions=4, threads=None):
    """The serving workload: n_jobs jobs of ranks log-uniform in [rank_lo,
    rank_hi] x GPUs per rank uniform in [1, gpus_hi]; each job's stream is
    made of batches whose record counts are log-uniform in [batch_lo,
    batch_hi] (one period of `period` batches, repeated shifted in time)."""
    rng = _rng(seed, 0, D_SHAPE, 7)
    ranks = np.clip(np.floor(np.exp(rng.uniform(math.log(rank_lo), math.log(rank_hi + 1), n_jobs))),
                    rank_lo, rank_hi).astype(np.int64)
    gpus = rng.integers(1, gpus_hi + 1, n_jobs)
    sizes = np.rint(np.exp(rng.uniform(math.log(batch_lo), math.log(batch_hi), (n_jobs, period)))).astype(np.int64)
    # events per GPU (and host intervals per rank) so one period holds the drawn records
    ev = np.maximum(1, np.ceil(sizes.sum(1) / (ranks * gpus + ranks)).astype(np.int64))

    def one(k):
        t = batched_trace_fast(k, ranks, gpus, ev, seed=seed, n_regions=n_regions)
        t.trace_id = k
        starts = np.sort(np.concatenate([t.host_se[:, 0], t.dev_se[:, 0]]))
        cum = np.cumsum(sizes[k])[:-1]
        cuts = starts[np.minimum(cum, starts.shape[0] - 1)]
        span = int(max(t.host_se[:, 1].max(), t.dev_se[:, 1].max() if t.n_dev else 0)) + 1
        return ServingJob(k, t, time_slices(t, cuts), span, n_regions)
    if threads is None:
        threads = min(32, os.cpu_count() or 1)
    return _pool_map(one, list(range(n_jobs)), threads)
