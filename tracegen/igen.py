"""Counter-based synthetic traces with a host (numpy) and a device (CUDA) twin.

Input generation only: nothing here computes any part of the reduction.
Every value is a pure function of (lane key, slot index, draw number)
through the SplitMix64 output function (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", 2014), and durations come from
integer inverse-CDF tables, so the two twins agree bit for bit and any lane
of a trace can be regenerated alone.  The device twin (csrc/igen.cu) makes
the full-size workloads in HBM at GPU speed; this module makes the same
lanes on the host for the oracle.

Lane layout (see csrc/igen.cu): a device lane of E events is S =
(7E + 5) // 10 kernel slots back to back (kernel, then an exponential gap;
the slot carries one copy, inside the kernel or in its gap, iff
((j+1) C) // S - (j C) // S == 1 with C = E - S), so records are in start
order by construction.  Kernel stream ids cycle over the lane's kernel
streams; all kernels of a device share one timeline at occupancy 0.7.
A host lane is H back-to-back intervals (state uniform over U / W / MPI,
exponential durations with means 50 / 5 / 10 us) plus one offload interval
up to the rank's end T = max(host end, last device end).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

from . import Trace, nested_regions

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libigen.so")
SRC = os.path.join(HERE, "csrc", "igen.cu")

M64 = (1 << 64) - 1
Q = 4096                      # table intervals (4097 entries)
DOM_HOST, DOM_DEV = 1, 2
LAW_LOGNORMAL, LAW_BIMODAL = 0, 1
MEAN_KERNEL_NS = {LAW_LOGNORMAL: 32974, LAW_BIMODAL: 100800}   # 20 us * e^0.5; 0.8 * 1 us + 0.2 * 500 us
HOST_MEAN_NS = np.array([50_000, 5_000, 10_000], np.int64)
CHUNK = 2048                  # slots per device chunk (igen_chunk_slots)

LANE_DTYPE = np.dtype([("key", "<u8"), ("out", "<u8"), ("n", "<u8"), ("t0", "<i8"), ("mean_gap", "<i8"),
                       ("chunk0", "<u4"), ("work_milli", "<u4"), ("is_host", "u1"), ("law", "u1"),
                       ("n_kstreams", "u1"), ("copy_stream0", "u1"), ("n_cstreams", "u1"), ("pad0", "u1"),
                       ("pad1", "u1"), ("pad2", "u1"), ("rank", "<u4"), ("pad3", "<u4")])
assert LANE_DTYPE.itemsize == 64


# ---------------------------------------------------------------- tables


def _tables():
    from scipy.special import ndtri
    q = (np.arange(Q + 1, dtype=np.float64) + 0.5) / (Q + 1)
    expo = np.rint(-np.log1p(-q) * 1e6).astype(np.int64)
    kern = np.maximum(np.rint(np.exp(math.log(20_000.0) + 1.0 * ndtri(q))), 1).astype(np.int64)
    copy = np.maximum(np.rint(np.exp(math.log(8_000.0) + 0.7 * ndtri(q))), 1).astype(np.int64)
    return kern, copy, expo


TAB_KERN, TAB_COPY, TAB_EXPO = _tables()


# ---------------------------------------------------------------- counters


def _mix_int(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def unit_key(seed: int, trace_id: int, domain: int, unit: int) -> int:
    k = _mix_int(seed ^ 0x6A09E667F3BCC909)
    k = _mix_int(k ^ (trace_id & M64))
    return _mix_int(k ^ ((domain << 40) & M64) ^ unit)


def unit_keys(seed: int, trace_id: int, domain: int, units: np.ndarray) -> np.ndarray:
    """unit_key over an array of units."""
    k = _mix_int(_mix_int(seed ^ 0x6A09E667F3BCC909) ^ (trace_id & M64))
    with np.errstate(over="ignore"):
        return _mix(np.uint64(k ^ ((domain << 40) & M64)) ^ units.astype(np.uint64))


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def draw(key: int, j: np.ndarray, t: int) -> np.ndarray:
    with np.errstate(over="ignore"):
        c = ((j.astype(np.uint64) << np.uint64(3)) | np.uint64(t)) * np.uint64(0xD6E8FEB86659FD93)
        return _mix(np.uint64(key) ^ c)


def tab(T: np.ndarray, u: np.ndarray) -> np.ndarray:
    i = (u >> np.uint64(52)).astype(np.int64)
    f = ((u >> np.uint64(36)) & np.uint64(0xFFFF)).astype(np.int64)
    return T[i] + (((T[i + 1] - T[i]) * f) >> 16)


# ---------------------------------------------------------------- specs


@dataclass
class TraceSpec:
    """Shape and laws of one generated trace."""
    trace_id: int
    seed: int
    devices_per_rank: np.ndarray      # uint32[n]
    dev_events: np.ndarray            # int64[m], rank-major
    host_events: np.ndarray           # int64[n] (intervals before the pad)
    work_milli: np.ndarray            # int64[n], kernel duration factor x 1000
    law: int = LAW_LOGNORMAL
    n_kstreams: int = 1
    copy_stream0: int = 0
    n_cstreams: int = 1
    n_regions: int = 1

    @property
    def n_ranks(self) -> int:
        return int(self.devices_per_rank.shape[0])

    @property
    def m_devices(self) -> int:
        return int(self.dev_events.shape[0])

    @property
    def n_records(self) -> int:
        return int(self.dev_events.sum() + self.host_events.sum() + self.n_ranks)

    def dev_rank(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_ranks), self.devices_per_rank.astype(np.int64))

    def mean_gap(self, rank: int) -> int:
        return MEAN_KERNEL_NS[self.law] * int(self.work_milli[rank]) * 3 // 7000

    def dev_key(self, g: int) -> int:
        return unit_key(self.seed, self.trace_id, DOM_DEV, g)

    def host_key(self, i: int) -> int:
        return unit_key(self.seed, self.trace_id, DOM_HOST, i)

    def offsets(self):
        dev_off = np.zeros(self.m_devices + 1, np.uint64)
        dev_off[1:] = np.cumsum(self.dev_events)
        host_off = np.zeros(self.n_ranks + 1, np.uint64)
        host_off[1:] = np.cumsum(self.host_events + 1)
        return host_off, dev_off


# ---------------------------------------------------------------- host twin


def _device_slots(spec: TraceSpec, g: int, j: np.ndarray):
    rank = int(spec.dev_rank()[g]) if spec.m_devices else 0
    key = spec.dev_key(g)
    u0 = draw(key, j, 0)
    if spec.law == LAW_LOGNORMAL:
        kd = tab(TAB_KERN, u0)
    else:
        kd = np.where((u0 >> np.uint64(11)) < np.uint64(7205759403792794), 1000, 500000).astype(np.int64)
    kd = np.maximum(kd * int(spec.work_milli[rank]) // 1000, 1)
    gap = tab(TAB_EXPO, draw(key, j, 1)) * spec.mean_gap(rank) // 1_000_000
    return key, kd, gap


def device_lane(spec: TraceSpec, g: int):
    """Records of device g: (se int64[E, 2], tag uint8[E])."""
    E = int(spec.dev_events[g])
    if E == 0:
        return np.zeros((0, 2), np.int64), np.zeros(0, np.uint8)
    S = (7 * E + 5) // 10
    C = E - S
    j = np.arange(S, dtype=np.int64)
    key, kd, gap = _device_slots(spec, g, j)
    ln = kd + gap
    ks = np.cumsum(ln) - ln
    e = j + (j * C) // S
    has = ((j + 1) * C) // S - (j * C) // S != 0
    se = np.empty((E, 2), np.int64)
    tag = np.empty(E, np.uint8)
    se[e, 0] = ks
    se[e, 1] = ks + kd
    tag[e] = (j % spec.n_kstreams).astype(np.uint8)
    jc = j[has]
    if jc.size:
        inside = (draw(key, jc, 2) >> np.uint64(32)) < np.uint64(1288490189)
        f = (draw(key, jc, 3) >> np.uint64(40)).astype(np.int64)
        kdc, gpc, ksc = kd[has], gap[has], ks[has]
        cs = np.where(inside, ksc + ((kdc * f) >> 24), ksc + kdc + ((gpc * f) >> 24))
        cd = np.maximum(tab(TAB_COPY, draw(key, jc, 4)), 1)
        kind = 1 + (draw(key, jc, 5) & np.uint64(1)).astype(np.int64)
        ec = e[has] + 1
        se[ec, 0] = cs
        se[ec, 1] = cs + cd
        tag[ec] = ((kind << 5) | (spec.copy_stream0 + jc % spec.n_cstreams)).astype(np.uint8)
    return se, tag


def device_lane_end(spec: TraceSpec, g: int) -> int:
    """Last end of device g's records (0 when it has none), computing the
    copies only where one can still end last."""
    E = int(spec.dev_events[g])
    if E == 0:
        return 0
    S = (7 * E + 5) // 10
    C = E - S
    j = np.arange(S, dtype=np.int64)
    key, kd, gap = _device_slots(spec, g, j)
    ln = kd + gap
    ks = np.cumsum(ln) - ln
    best = int((ks + kd).max())
    # a copy of slot j starts before ks[j] + ln[j] and lasts at most the table maximum
    cand = (ks + ln + int(TAB_COPY[-1]) > best) & ((((j + 1) * C) // S - (j * C) // S) != 0)
    jc = j[cand]
    if jc.size:
        inside = (draw(key, jc, 2) >> np.uint64(32)) < np.uint64(1288490189)
        f = (draw(key, jc, 3) >> np.uint64(40)).astype(np.int64)
        cs = np.where(inside, ks[cand] + ((kd[cand] * f) >> 24), ks[cand] + kd[cand] + ((gap[cand] * f) >> 24))
        cd = np.maximum(tab(TAB_COPY, draw(key, jc, 4)), 1)
        best = max(best, int((cs + cd).max()))
    return best


def host_lane(spec: TraceSpec, i: int):
    """Host intervals of rank i without the closing pad: (se, state, end)."""
    H = int(spec.host_events[i])
    key = spec.host_key(i)
    j = np.arange(H, dtype=np.int64)
    state = ((draw(key, j, 0) >> np.uint64(32)) % np.uint64(3)).astype(np.int64)
    dur = tab(TAB_EXPO, draw(key, j, 1)) * HOST_MEAN_NS[state] // 1_000_000
    end = np.cumsum(dur)
    se = np.empty((H, 2), np.int64)
    se[:, 0] = end - dur
    se[:, 1] = end
    return se, state.astype(np.uint8), int(end[-1]) if H else 0


def rank_ends(spec: TraceSpec, threads=None) -> np.ndarray:
    """T_i = max(host end, last device end of rank i, 1) for every rank."""
    if threads is None:
        threads = min(32, os.cpu_count() or 1)
    dr = spec.dev_rank()
    with ThreadPoolExecutor(threads) as ex:
        dev_end = list(ex.map(lambda g: device_lane_end(spec, g), range(spec.m_devices)))
        host_end = list(ex.map(lambda i: host_lane(spec, i)[2], range(spec.n_ranks)))
    T = np.maximum(np.asarray(host_end, np.int64), 1)
    for g, e in enumerate(dev_end):
        T[dr[g]] = max(T[dr[g]], e)
    return T


def host_trace(spec: TraceSpec, T=None, ranks=None) -> Trace:
    """The whole trace (or the block of ranks `ranks`, with the windows of the
    whole trace) made on the host."""
    if T is None:
        T = rank_ends(spec)
    win_all = nested_regions(T, spec.n_regions)
    ranks = np.arange(spec.n_ranks) if ranks is None else np.asarray(ranks, np.int64)
    first_dev = np.concatenate([[0], np.cumsum(spec.devices_per_rank.astype(np.int64))])
    hs, hst, hcnt, ds, dtg, dcnt, dpr = [], [], [], [], [], [], []
    for i in ranks:
        se, st, end = host_lane(spec, int(i))
        se = np.concatenate([se, np.array([[end, max(int(T[i]), end)]], np.int64)])
        st = np.concatenate([st, np.array([1], np.uint8)])
        hs.append(se)
        hst.append(st)
        hcnt.append(se.shape[0])
        dpr.append(int(spec.devices_per_rank[i]))
        for g in range(int(first_dev[i]), int(first_dev[i + 1])):
            a, b = device_lane(spec, g)
            ds.append(a)
            dtg.append(b)
            dcnt.append(a.shape[0])
    host_off = np.zeros(len(hcnt) + 1, np.uint64)
    host_off[1:] = np.cumsum(hcnt)
    dev_off = np.zeros(len(dcnt) + 1, np.uint64)
    dev_off[1:] = np.cumsum(dcnt)
    return Trace(trace_id=spec.trace_id, n_ranks=len(ranks), devices_per_rank=np.asarray(dpr, np.uint32),
                 region_window=np.ascontiguousarray(win_all[:, ranks]),
                 host_se=np.concatenate(hs) if hs else np.zeros((0, 2), np.int64),
                 host_state=np.concatenate(hst) if hst else np.zeros(0, np.uint8), host_off=host_off,
                 dev_se=np.concatenate(ds) if ds else np.zeros((0, 2), np.int64),
                 dev_tag=np.concatenate(dtg) if dtg else np.zeros(0, np.uint8), dev_off=dev_off,
                 sorted_by_start=True, meta=dict(workload="igen", ranks=ranks))


# ---------------------------------------------------------------- device twin

_lib = None


def build(force=False) -> str:
    """Compile csrc/igen.cu into libigen.so (sm_103a)."""
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC):
        return LIB_PATH
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
           "-std=c++17", "-Xcompiler", "-fPIC", "-cudart=shared", "-shared", "-o", tmp, SRC,
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        U32 = ctypes.c_uint32
        lib.igen_generate.argtypes = [P, U32, P, U32, P, P, P, P, P, P, P, P, P, P, P, P, P, U32, P, P]
        lib.igen_generate.restype = ctypes.c_int
        lib.igen_chunk_slots.restype = ctypes.c_int
        assert lib.igen_chunk_slots() == CHUNK
        _lib = lib
    return _lib


@dataclass
class DeviceTrace:
    """A generated trace in HBM: header arrays on the host, record tensors on
    the device (views into the wave's buffers, 16-byte aligned)."""
    trace_id: int
    n_ranks: int
    devices_per_rank: np.ndarray
    region_window: np.ndarray
    host_off: np.ndarray
    dev_off: np.ndarray
    host_se: object
    host_state: object
    dev_se: object
    dev_tag: object
    T: np.ndarray

    @property
    def n_regions(self) -> int:
        return int(self.region_window.shape[0])

    @property
    def n_records(self) -> int:
        return int(self.host_off[-1] + self.dev_off[-1])


def generate_device(specs, device=0, stream=None):
    """Generate every trace of `specs` on the GPU in one pass.  Returns
    [DeviceTrace] (record tensors share four wave buffers)."""
    import torch
    lib = _load()
    dev = torch.device("cuda", device)
    up = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    parts, chunk_lane = [], []
    rank_host, rank_dev0, rank_ndev = [], [], []
    dbase, hbase = [], []
    drow = hrow = 0
    nlane = nchunk = 0
    for sp in specs:
        host_off, dev_off = sp.offsets()
        drow = (drow + 15) // 16 * 16
        hrow = (hrow + 15) // 16 * 16
        dbase.append(drow)
        hbase.append(hrow)
        m, n = sp.m_devices, sp.n_ranks
        dr = sp.dev_rank()
        L = np.zeros(m + n, LANE_DTYPE)
        L["key"][:m] = unit_keys(sp.seed, sp.trace_id, DOM_DEV, np.arange(m))
        L["key"][m:] = unit_keys(sp.seed, sp.trace_id, DOM_HOST, np.arange(n))
        L["out"][:m] = drow + dev_off[:-1].astype(np.int64)
        L["out"][m:] = hrow + host_off[:-1].astype(np.int64)
        L["n"][:m] = sp.dev_events
        L["n"][m:] = sp.host_events
        L["mean_gap"][:m] = MEAN_KERNEL_NS[sp.law] * sp.work_milli[dr] * 3 // 7000
        L["work_milli"][:m] = sp.work_milli[dr]
        L["is_host"][m:] = 1
        L["law"][:m] = sp.law
        L["n_kstreams"][:m] = sp.n_kstreams
        L["copy_stream0"][:m] = sp.copy_stream0
        L["n_cstreams"][:m] = sp.n_cstreams
        L["rank"][:m] = dr
        L["rank"][m:] = np.arange(n)
        slots = np.concatenate([(7 * sp.dev_events + 5) // 10, sp.host_events]).astype(np.int64)
        nc = (slots + CHUNK - 1) // CHUNK
        c0 = nchunk + np.concatenate([[0], np.cumsum(nc)[:-1]])
        L["chunk0"] = c0
        chunk_lane.append(np.repeat(np.arange(nlane, nlane + m + n, dtype=np.uint32), nc))
        nchunk += int(nc.sum())
        first_dev = np.concatenate([[0], np.cumsum(sp.devices_per_rank.astype(np.int64))])
        rank_host.append(nlane + m + np.arange(n))
        rank_dev0.append(nlane + first_dev[:-1])
        rank_ndev.append(sp.devices_per_rank.astype(np.int64))
        parts.append(L)
        nlane += m + n
        drow += int(dev_off[-1])
        hrow += int(host_off[-1])
    lanes_np = np.concatenate(parts) if parts else np.zeros(0, LANE_DTYPE)
    cl = np.concatenate(chunk_lane) if chunk_lane else np.zeros(0, np.uint32)
    rank_host = np.concatenate(rank_host) if rank_host else np.zeros(0, np.int64)
    rank_dev0 = np.concatenate(rank_dev0) if rank_dev0 else np.zeros(0, np.int64)
    rank_ndev = np.concatenate(rank_ndev) if rank_ndev else np.zeros(0, np.int64)
    lanes = lanes_np
    d_lanes = up(lanes_np.view(np.uint8))
    d_cl = up(cl.astype(np.uint32).view(np.int32)) if cl.size else torch.zeros(1, dtype=torch.int32, device=dev)
    tk, tc, te = up(TAB_KERN), up(TAB_COPY), up(TAB_EXPO)
    sums = torch.empty(max(nchunk, 1), dtype=torch.int64, device=dev)
    base = torch.empty_like(sums)
    lane_end = torch.empty(max(len(lanes), 1), dtype=torch.int64, device=dev)
    dse = torch.empty((max(drow, 1), 2), dtype=torch.int64, device=dev)
    dtag = torch.empty(max(drow, 16), dtype=torch.uint8, device=dev)
    hse = torch.empty((max(hrow, 1), 2), dtype=torch.int64, device=dev)
    hst = torch.empty(max(hrow, 16), dtype=torch.uint8, device=dev)
    rh, rd0, rnd = (up(np.asarray(x, np.uint32).view(np.int32)) if len(x) else torch.zeros(1, dtype=torch.int32, device=dev)
                    for x in (rank_host, rank_dev0, rank_ndev))
    T = torch.empty(max(len(rank_host), 1), dtype=torch.int64, device=dev)
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    rc = lib.igen_generate(d_lanes.data_ptr(), len(lanes), d_cl.data_ptr(), nchunk, tk.data_ptr(), tc.data_ptr(),
                           te.data_ptr(), sums.data_ptr(), base.data_ptr(), lane_end.data_ptr(), dse.data_ptr(),
                           dtag.data_ptr(), hse.data_ptr(), hst.data_ptr(), rh.data_ptr(), rd0.data_ptr(),
                           rnd.data_ptr(), len(rank_host), T.data_ptr(), ctypes.c_void_p(s))
    if rc != 0:
        raise RuntimeError(f"igen_generate failed with CUDA error {rc}")
    torch.cuda.current_stream(dev).synchronize() if stream is None else stream.synchronize()
    T_host = T.cpu().numpy()
    out = []
    r0 = 0
    for k, sp in enumerate(specs):
        host_off, dev_off = sp.offsets()
        Tk = T_host[r0:r0 + sp.n_ranks].copy()
        r0 += sp.n_ranks
        nd, nh = int(dev_off[-1]), int(host_off[-1])
        out.append(DeviceTrace(trace_id=sp.trace_id, n_ranks=sp.n_ranks, devices_per_rank=sp.devices_per_rank,
                               region_window=nested_regions(Tk, sp.n_regions), host_off=host_off, dev_off=dev_off,
                               host_se=hse[hbase[k]:hbase[k] + nh], host_state=hst[hbase[k]:hbase[k] + nh],
                               dev_se=dse[dbase[k]:dbase[k] + nd], dev_tag=dtag[dbase[k]:dbase[k] + nd], T=Tk))
    del sums, base, lane_end
    return out


# ---------------------------------------------------------------- workloads


def _rng(seed, k):
    return np.random.default_rng([seed, k])


def scale_spec(seed=0x7A1F + 3, scale=1.0, trace_id=3, n_ranks=1024, gpus_per_rank=4, n_regions=4) -> TraceSpec:
    """The scale workload: 1024 ranks x 4 GPUs x 8 streams (kernels on streams
    0-5, copies on 6-7), bimodal kernels (1 us / 500 us, 80/20), 20% of the
    ranks (a seeded permutation) with 1.5x events, 222k device events per GPU
    and 100k host intervals per rank at scale 1, 4 nested regions."""
    base = max(1, int(round(222_000 * scale)))
    host = max(1, int(round(100_000 * scale)))
    rng = _rng(seed, 1)
    heavy = np.zeros(n_ranks, bool)
    heavy[rng.permutation(n_ranks)[: int(round(0.2 * n_ranks))]] = True
    per_rank = np.where(heavy, int(round(1.5 * base)), base).astype(np.int64)
    return TraceSpec(trace_id=trace_id, seed=seed, devices_per_rank=np.full(n_ranks, gpus_per_rank, np.uint32),
                     dev_events=np.repeat(per_rank, gpus_per_rank), host_events=np.full(n_ranks, host, np.int64),
                     work_milli=np.full(n_ranks, 1000, np.int64), law=LAW_BIMODAL, n_kstreams=6, copy_stream0=6,
                     n_cstreams=2, n_regions=n_regions)


def batched_specs(n_traces=4096, seed=0x7A1F + 2, ev_lo=1_000, ev_hi=1_000_000, max_ranks=512, max_gpus=8,
                  n_regions=8) -> list:
    """The batched workload: ranks log-uniform in [1, max_ranks], GPUs per
    rank uniform in [1, max_gpus], events per GPU (= host intervals per rank)
    log-uniform in [ev_lo, ev_hi], lognormal kernels on one stream, rank work
    factors uniform in [0.7, 1.0], 8 nested regions."""
    rng = _rng(seed, 2)
    ranks = np.clip(np.floor(np.exp(rng.uniform(0, math.log(max_ranks + 1), n_traces))), 1, max_ranks).astype(np.int64)
    gpus = rng.integers(1, max_gpus + 1, n_traces)
    ev = np.clip(np.rint(np.exp(rng.uniform(math.log(ev_lo), math.log(ev_hi), n_traces))), ev_lo, ev_hi).astype(np.int64)
    out = []
    for k in range(n_traces):
        n, g, e = int(ranks[k]), int(gpus[k]), int(ev[k])
        work = 700 + _rng(seed, 1000 + k).integers(0, 301, n)
        out.append(TraceSpec(trace_id=k, seed=seed, devices_per_rank=np.full(n, g, np.uint32),
                             dev_events=np.full(n * g, e, np.int64), host_events=np.full(n, e, np.int64),
                             work_milli=work.astype(np.int64), law=LAW_LOGNORMAL, n_kstreams=1, copy_stream0=0,
                             n_cstreams=1, n_regions=n_regions))
    return out


def waves(specs, max_records: int) -> list:
    """Consecutive groups of whole traces of at most max_records records
    each (a trace larger than that forms a wave of its own)."""
    out, cur, n = [], [], 0
    for sp in specs:
        r = sp.n_records
        if cur and n + r > max_records:
            out.append(cur)
            cur, n = [], 0
        cur.append(sp)
        n += r
    if cur:
        out.append(cur)
    return out
