"""Native client load of the serving workload (csrc/serve_load.cc).

Submitter threads with Poisson arrivals and query threads with a fixed query
period, all in native threads that call the library's C ABI directly, so the
client-side query latency holds no interpreter time.  The caller passes the
library's `talp_gpu_server_submit` and `talp_gpu_server_query` entry points
and its jobs' slices as `talp_gpu_trace_batch` records (addresses); this
module knows nothing of the library beyond the header's C types.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "serve_load.cc")
LIB_PATH = os.path.join(HERE, "libserve_load.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")


class SlJob(ctypes.Structure):
    _fields_ = [("job_id", ctypes.c_uint64), ("n_ranks", ctypes.c_uint32), ("n_devices", ctypes.c_uint32),
                ("n_slices", ctypes.c_uint32), ("n_regions", ctypes.c_uint32), ("span", ctypes.c_int64),
                ("slices", ctypes.c_void_p)]


class SlConfig(ctypes.Structure):
    _fields_ = [("rate", ctypes.c_double), ("query_s", ctypes.c_double), ("seconds", ctypes.c_double),
                ("n_sub", ctypes.c_uint32), ("n_q", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class SlResult(ctypes.Structure):
    _fields_ = [("slices", ctypes.c_uint64), ("records", ctypes.c_uint64), ("queries", ctypes.c_uint64),
                ("errors", ctypes.c_uint64), ("first_error", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("wall_s", ctypes.c_double)]


_lib = None


def build(force=False) -> str:
    """Compile csrc/serve_load.cc into libserve_load.so (host code only)."""
    deps = [SRC, os.path.join(INCLUDE, "talp_gpu.h")]
    if not force and os.path.exists(LIB_PATH) and all(os.path.getmtime(LIB_PATH) >= os.path.getmtime(p) for p in deps):
        return LIB_PATH
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-I", INCLUDE, "-o", tmp, SRC])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.sl_run.argtypes = [P, P, P, ctypes.POINTER(SlJob), ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                               ctypes.POINTER(SlConfig), ctypes.POINTER(ctypes.c_double), ctypes.c_uint64,
                               ctypes.POINTER(SlResult)]
        lib.sl_run.restype = ctypes.c_int
        _lib = lib
    return _lib


def run(server, submit_fn, query_fn, jobs, next_q, rate, query_s, seconds, n_sub=8, n_q=16, seed=7):
    """Run the load for `seconds` against `server` (a talp_gpu_server*).

    jobs: list of dicts with job_id, n_ranks, n_devices, n_regions, span and
    slices (the address of an array of talp_gpu_trace_batch records, host
    record arrays, kept alive by the caller) and n_slices.  next_q: each
    job's next slice number, advanced in place.  Returns the query
    latencies (seconds) and the counts."""
    lib = _load()
    if isinstance(server, ctypes.c_void_p):
        server = server.value
    arr = (SlJob * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i] = SlJob(j["job_id"], j["n_ranks"], j["n_devices"], j["n_slices"], j["n_regions"], j["span"],
                       j["slices"])
    nq = (ctypes.c_uint64 * len(jobs))(*[int(x) for x in next_q])
    cfg = SlConfig(float(rate), float(query_s), float(seconds), n_sub, n_q, seed)
    cap = int(seconds / query_s + 2) * len(jobs) * 2 + 1024
    lat = np.zeros(cap, np.float64)
    res = SlResult()
    rc = lib.sl_run(ctypes.c_void_p(server), ctypes.c_void_p(submit_fn), ctypes.c_void_p(query_fn), arr, len(jobs),
                    nq, ctypes.byref(cfg), lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cap,
                    ctypes.byref(res))
    if rc != 0:
        raise ValueError("sl_run: bad arguments")
    for i in range(len(jobs)):
        next_q[i] = int(nq[i])
    n = min(int(res.queries), cap)
    return {"lat": lat[:n].tolist(), "slices": int(res.slices), "records": int(res.records),
            "queries": int(res.queries), "errors": int(res.errors), "first_error": int(res.first_error),
            "wall_s": float(res.wall_s)}
