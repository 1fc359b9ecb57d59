"""CPU oracle (test infrastructure only).

The plain C statement of the extended POP metrics lives in talp_oracle.c; this
module compiles it with gcc (no FMA contraction) and wraps it with ctypes.
Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
it; the product library never imports it.

Inputs are numpy arrays in the record layout of the trace generator:
host_se int64[N,2], host_state uint8[N], host_off uint64[n+1],
dev_se int64[N,2], dev_tag uint8[N], dev_off uint64[m+1],
devices_per_rank uint32[n], region_window int64[R,n,2].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from types import SimpleNamespace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "talp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

INT_FIELDS = ("elapsed_ns", "sum_useful", "sum_offload", "sum_mpi", "max_useful_offload",
              "sum_kernel", "max_kernel", "max_busy", "sum_mem", "sum_idle", "sum_hidden_mem")
RATIO_FIELDS = ("host_pe", "host_mpi_pe", "host_mpi_lb", "host_mpi_ce", "host_oe",
                "dev_pe", "dev_lb", "dev_ce", "dev_oe")
FLAG_EMPTY, FLAG_HOST_NOT_TILED, FLAG_NO_DEVICES = 1, 2, 4
THREAD_INT_FIELDS = ("elapsed_ns", "sum_useful", "sum_offload", "sum_busiest", "max_busiest", "n_threads")
THREAD_RATIO_FIELDS = ("pe", "mpi_pe", "mpi_lb", "mpi_ce", "thread_lb", "oe")


def compile_c(src: str, out: str) -> str:
    """gcc -O2, FP contraction off, so every product and quotient rounds once."""
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-o", tmp, src])
    os.replace(tmp, out)
    return out


def build(force=False) -> str:
    """Compile the oracle shared library next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(SOURCE):
        compile_c(SOURCE, _LIB)
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Oracle:
    """ctypes view of one build of talp_oracle.c."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        P = ctypes.c_void_p
        lib.oracle_validate.argtypes = [ctypes.c_uint64, P, P, ctypes.c_uint64, P, P]
        lib.oracle_validate.restype = ctypes.c_int
        lib.oracle_host_sums.argtypes = [ctypes.c_uint32, P, P, P, P, P]
        lib.oracle_host_sums.restype = None
        lib.oracle_device_unions.argtypes = [ctypes.c_uint32, P, P, P, P, P, P]
        lib.oracle_device_unions.restype = ctypes.c_int
        lib.oracle_metrics.argtypes = [ctypes.c_uint32, P, P, P, P, P, P, P]
        lib.oracle_metrics.restype = None
        lib.oracle_concurrency.argtypes = [ctypes.c_uint32, P, P, P, P, P, ctypes.c_uint32, P]
        lib.oracle_concurrency.restype = ctypes.c_int
        lib.oracle_scalability.argtypes = [ctypes.c_uint32, P, P, P, ctypes.c_uint32, ctypes.c_int, P]
        lib.oracle_scalability.restype = None
        lib.oracle_thread_metrics.argtypes = [ctypes.c_uint32, P, P, P, P, P]
        lib.oracle_thread_metrics.restype = None
        self.lib = lib

    def validate(self, t) -> int:
        hse, hst = _c(t.host_se, np.int64), _c(t.host_state, np.uint8)
        dse, dtg = _c(t.dev_se, np.int64), _c(t.dev_tag, np.uint8)
        return int(self.lib.oracle_validate(hse.shape[0], _p(hse), _p(hst), dse.shape[0], _p(dse), _p(dtg)))

    def host_sums(self, t, region: int) -> np.ndarray:
        """int64[n,3]: per rank (useful, offload, MPI) time inside the region."""
        n = int(t.n_ranks)
        out = np.zeros((n, 3), np.int64)
        hse, hst, hoff = _c(t.host_se, np.int64), _c(t.host_state, np.uint8), _c(t.host_off, np.uint64)
        win = _c(t.region_window[region], np.int64)
        self.lib.oracle_host_sums(n, _p(hse), _p(hst), _p(hoff), _p(win), _p(out))
        return out

    def device_unions(self, t, region: int) -> np.ndarray:
        """int64[m,3]: per device |U kernels|, |U memory ops|, |U all| inside the region."""
        n = int(t.n_ranks)
        dpr = _c(t.devices_per_rank, np.uint32)
        m = int(dpr.sum())
        out = np.zeros((m, 3), np.int64)
        dse, dtg, doff = _c(t.dev_se, np.int64), _c(t.dev_tag, np.uint8), _c(t.dev_off, np.uint64)
        win = _c(t.region_window[region], np.int64)
        rc = self.lib.oracle_device_unions(n, _p(dpr), _p(dse), _p(dtg), _p(doff), _p(win), _p(out))
        if rc != 0:
            raise MemoryError("oracle_device_unions")
        return out

    def concurrency(self, t, region: int, K: int = 8) -> np.ndarray:
        """int64[m, 2, K]: per device, time with at least k active records
        (all records, then kernels only), k = 1 .. K, inside the region."""
        n = int(t.n_ranks)
        dpr = _c(t.devices_per_rank, np.uint32)
        m = int(dpr.sum())
        out = np.zeros((m, 2, K), np.int64)
        dse, dtg, doff = _c(t.dev_se, np.int64), _c(t.dev_tag, np.uint8), _c(t.dev_off, np.uint64)
        win = _c(t.region_window[region], np.int64)
        if self.lib.oracle_concurrency(n, _p(dpr), _p(dse), _p(dtg), _p(doff), _p(win), K, _p(out)) != 0:
            raise MemoryError("oracle_concurrency")
        return out

    def scalability(self, runs, ref: int = 0, weak: bool = False) -> list:
        """Scaling factors of region-metrics dicts `runs` (one per run, as
        region_metrics returns) against runs[ref]: per run a dict with
        speedup, host_comp_scal, host_global_eff, dev_comp_scal, dev_global_eff."""
        k = len(runs)
        iruns = np.array([[r["elapsed_ns"], r["sum_useful"], r["sum_kernel"]] for r in runs], np.int64)
        units = np.array([[r["n_ranks"], r["m_devices"]] for r in runs], np.uint32)
        pe = np.array([[r["host_pe"], r["dev_pe"]] for r in runs], np.float64)
        out = np.zeros((k, 5), np.float64)
        self.lib.oracle_scalability(k, _p(iruns), _p(units), _p(pe), int(ref), int(bool(weak)), _p(out))
        names = ("speedup", "host_comp_scal", "host_global_eff", "dev_comp_scal", "dev_global_eff")
        return [{nm: float(v) for nm, v in zip(names, row)} for row in out]

    def thread_metrics_from_sums(self, proc_off, hs) -> dict:
        """Host tree with threads from per-thread sums hs int64[nT, 3] (the
        units of process i are proc_off[i] .. proc_off[i+1]-1)."""
        po = _c(proc_off, np.uint32)
        hs = _c(hs, np.int64)
        assert po[0] == 0 and po[-1] == hs.shape[0] and np.all(np.diff(po.astype(np.int64)) >= 1)
        iout = np.zeros(6, np.int64)
        dout = np.zeros(6, np.float64)
        flags = np.zeros(1, np.uint32)
        self.lib.oracle_thread_metrics(po.shape[0] - 1, _p(po), _p(hs), _p(iout), _p(dout), _p(flags))
        res = {k: int(v) for k, v in zip(THREAD_INT_FIELDS, iout)}
        res.update({k: float(v) for k, v in zip(THREAD_RATIO_FIELDS, dout)})
        res["flags"] = int(flags[0])
        res["n_procs"] = int(po.shape[0] - 1)
        return res

    def thread_metrics(self, t, region: int, proc_off) -> dict:
        """Host tree with threads of one region: every host unit of t is a
        thread, grouped into processes by proc_off."""
        return self.thread_metrics_from_sums(proc_off, self.host_sums(t, region))

    def metrics_from_sums(self, n_ranks, devices_per_rank, hs, du, win) -> dict:
        dpr = _c(devices_per_rank, np.uint32)
        hs = _c(hs, np.int64)
        du = _c(du, np.int64)
        win = _c(win, np.int64)
        iout = np.zeros(11, np.int64)
        dout = np.zeros(9, np.float64)
        flags = np.zeros(1, np.uint32)
        self.lib.oracle_metrics(int(n_ranks), _p(dpr), _p(hs), _p(du), _p(win), _p(iout), _p(dout), _p(flags))
        res = {k: int(v) for k, v in zip(INT_FIELDS, iout)}
        res.update({k: float(v) for k, v in zip(RATIO_FIELDS, dout)})
        res["flags"] = int(flags[0])
        res["n_ranks"] = int(n_ranks)
        res["m_devices"] = int(dpr.sum())
        return res

    def region_metrics(self, t, region: int) -> dict:
        """All sums and the nine ratios of one region (Eqs. 1, 6-12)."""
        hs = self.host_sums(t, region)
        du = self.device_unions(t, region)
        return self.metrics_from_sums(t.n_ranks, t.devices_per_rank, hs, du, t.region_window[region])

    def trace_metrics(self, t) -> list:
        return [self.region_metrics(t, r) for r in range(int(t.region_window.shape[0]))]


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def validate(t):
    return default().validate(t)


def host_sums(t, region):
    return default().host_sums(t, region)


def device_unions(t, region):
    return default().device_unions(t, region)


def metrics_from_sums(*a):
    return default().metrics_from_sums(*a)


def concurrency(t, region, K=8):
    return default().concurrency(t, region, K)


def scalability(runs, ref=0, weak=False):
    return default().scalability(runs, ref, weak)


def region_metrics(t, region):
    return default().region_metrics(t, region)


def thread_metrics(t, region, proc_off):
    return default().thread_metrics(t, region, proc_off)


def trace_metrics(t):
    return default().trace_metrics(t)


def device_unions_by_rank(fetch, n_ranks, devices_per_rank, region_window, block_ranks=64, threads=None):
    """int64[R, m, 3]: oracle_device_unions of every region for every device
    of a trace too large to hold on the host at once.  fetch(r0, r1) returns
    (dev_se, dev_tag, dev_off) of ranks r0 .. r1-1 (dev_off from 0 over their
    devices); blocks of ranks are fetched in turn and their ranks reduced by
    the oracle on host threads (the C calls release the GIL).  Plumbing only:
    every number comes from oracle_device_unions, one rank at a time."""
    dpr = np.asarray(devices_per_rank, np.int64)
    win = np.asarray(region_window, np.int64)
    R, m = int(win.shape[0]), int(dpr.sum())
    first = np.concatenate([[0], np.cumsum(dpr)])
    out = np.zeros((R, m, 3), np.int64)
    threads = threads or os.cpu_count() or 1
    orc = default()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        for r0 in range(0, int(n_ranks), block_ranks):
            r1 = min(int(n_ranks), r0 + block_ranks)
            se, tag, off = fetch(r0, r1)
            off = np.asarray(off, np.uint64)

            def job(i, se=se, tag=tag, off=off, r0=r0):
                g0, g1 = int(first[i] - first[r0]), int(first[i + 1] - first[r0])
                a, b = int(off[g0]), int(off[g1])
                one = SimpleNamespace(n_ranks=1, devices_per_rank=dpr[i:i + 1].astype(np.uint32),
                                      dev_se=se[a:b], dev_tag=tag[a:b],
                                      dev_off=(off[g0:g1 + 1] - off[g0]).astype(np.uint64),
                                      region_window=win[:, i:i + 1])
                return i, [orc.device_unions(one, r) for r in range(R)]

            for i, res in ex.map(job, range(r0, r1)):
                for r in range(R):
                    out[r, first[i]:first[i + 1]] = res[r]
    return out
