"""Shared test helpers: golden fixtures -> traces, brute-force tick counting."""
import glob
import json
import os

import numpy as np

from tracegen import Trace, make_tag

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pils_cases():
    return sorted(glob.glob(os.path.join(GOLDEN, "pils_*.json")))


def load_fixture(path):
    return json.load(open(path))


def fixture_trace(fx, trace_id=0):
    """Build a trace from a golden fixture (device records sorted by start)."""
    n = fx["n_ranks"]
    dpr = np.asarray(fx["devices_per_rank"], np.uint32)
    win = np.asarray([fx["window"]], np.int64)            # one region
    hse, hst, hoff = [], [], [0]
    for i in range(n):
        rows = fx["host"][i]
        for s, e, q in rows:
            hse.append((s, e))
            hst.append(q)
        hoff.append(hoff[-1] + len(rows))
    dse, dtg, doff = [], [], [0]
    for g in range(int(dpr.sum())):
        rows = sorted(fx["device"][g], key=lambda r: r[0])
        for s, e, kind, stream in rows:
            dse.append((s, e))
            dtg.append(int(make_tag(kind, stream)))
        doff.append(doff[-1] + len(rows))
    return Trace(trace_id=trace_id, n_ranks=n, devices_per_rank=dpr, region_window=win,
                 host_se=np.asarray(hse, np.int64).reshape(-1, 2), host_state=np.asarray(hst, np.uint8),
                 host_off=np.asarray(hoff, np.uint64),
                 dev_se=np.asarray(dse, np.int64).reshape(-1, 2), dev_tag=np.asarray(dtg, np.uint8),
                 dev_off=np.asarray(doff, np.uint64))


def tick_device(trace, region):
    """Per device, count the nanoseconds covered by kernels, by memory
    operations and by either, inside the rank window (one boolean per ns)."""
    out = []
    win = trace.region_window[region]
    g = 0
    for i in range(trace.n_ranks):
        a, b = int(win[i, 0]), int(win[i, 1])
        for _ in range(int(trace.devices_per_rank[i])):
            lo, hi = int(trace.dev_off[g]), int(trace.dev_off[g + 1])
            if b <= a:
                out.append((0, 0, 0))
                g += 1
                continue
            cov_k = np.zeros(b - a, bool)
            cov_m = np.zeros(b - a, bool)
            for j in range(lo, hi):
                s, e = int(trace.dev_se[j, 0]), int(trace.dev_se[j, 1])
                ticks = np.arange(s, e)
                ticks = ticks[(ticks >= a) & (ticks < b)] - a
                if (int(trace.dev_tag[j]) >> 5) == 0:
                    cov_k[ticks] = True
                else:
                    cov_m[ticks] = True
            out.append((int(cov_k.sum()), int(cov_m.sum()), int((cov_k | cov_m).sum())))
            g += 1
    return np.asarray(out, np.int64).reshape(-1, 3)


def tick_concurrency(trace, region, K):
    """Per device, count the nanoseconds with at least k active records
    (all kinds, then kernels only), k = 1 .. K, inside the rank window: one
    counter per ns."""
    win = trace.region_window[region]
    m = int(np.asarray(trace.devices_per_rank).sum())
    out = np.zeros((m, 2, K), np.int64)
    g = 0
    for i in range(trace.n_ranks):
        a, b = int(win[i, 0]), int(win[i, 1])
        for _ in range(int(trace.devices_per_rank[i])):
            lo, hi = int(trace.dev_off[g]), int(trace.dev_off[g + 1])
            if b > a:
                cnt = np.zeros((2, b - a), np.int64)
                for j in range(lo, hi):
                    s, e = max(int(trace.dev_se[j, 0]), a), min(int(trace.dev_se[j, 1]), b)
                    if e > s:
                        cnt[0, s - a:e - a] += 1
                        if (int(trace.dev_tag[j]) >> 5) == 0:
                            cnt[1, s - a:e - a] += 1
                for k in range(1, K + 1):
                    out[g, :, k - 1] = (cnt >= k).sum(axis=1)
            g += 1
    return out


def tick_host(trace, region):
    """Per rank and state, the number of nanosecond ticks of each host
    interval that fall inside the window, summed over intervals."""
    win = trace.region_window[region]
    out = np.zeros((trace.n_ranks, 3), np.int64)
    for i in range(trace.n_ranks):
        a, b = int(win[i, 0]), int(win[i, 1])
        for j in range(int(trace.host_off[i]), int(trace.host_off[i + 1])):
            s, e = int(trace.host_se[j, 0]), int(trace.host_se[j, 1])
            ticks = np.arange(s, e)
            out[i, int(trace.host_state[j])] += int(np.count_nonzero((ticks >= a) & (ticks < b)))
    return out


def host_tiles_windows(trace, region):
    """True if each rank's host intervals exactly tile its window."""
    win = trace.region_window[region]
    for i in range(trace.n_ranks):
        a, b = int(win[i, 0]), int(win[i, 1])
        se = trace.host_se[int(trace.host_off[i]):int(trace.host_off[i + 1])]
        if b <= a:
            return False
        cov = np.zeros(b - a, np.int32)
        for s, e in se:
            lo, hi = max(int(s), a), min(int(e), b)
            if hi > lo:
                cov[lo - a:hi - a] += 1
        if not np.all(cov == 1):
            return False
    return True


def host_units_trace(trace, order, trace_id=0):
    """A device-free trace whose host unit k is unit order[k] of `trace` (its
    intervals and windows); units may repeat."""
    order = [int(u) for u in order]
    segs = [trace.host_segment(u) for u in order]
    hoff = np.zeros(len(order) + 1, np.uint64)
    hoff[1:] = np.cumsum([s[0].shape[0] for s in segs])
    return Trace(trace_id=trace_id, n_ranks=len(order), devices_per_rank=np.zeros(len(order), np.uint32),
                 region_window=np.ascontiguousarray(trace.region_window[:, order, :]),
                 host_se=np.concatenate([s[0] for s in segs]).reshape(-1, 2).astype(np.int64),
                 host_state=np.concatenate([s[1] for s in segs]).astype(np.uint8), host_off=hoff,
                 dev_se=np.zeros((0, 2), np.int64), dev_tag=np.zeros(0, np.uint8),
                 dev_off=np.zeros(1, np.uint64))
