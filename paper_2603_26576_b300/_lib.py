"""ctypes binding of include/talp_gpu.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtalp_gpu.so")

TALP_GPU_MAX_REGIONS = 8
TALP_GPU_ALL = (1 << 64) - 1
TALP_GPU_ALL_REGIONS = (1 << 32) - 1
TALP_GPU_DEVICE_PTRS = 0x1
TALP_GPU_SORTED_BY_START = 0x2
TALP_GPU_APPEND = 0x4
TALP_GPU_HOLD_BACK = 0x8
TALP_GPU_NOT_SORTED = 0x10
TALP_GPU_GROUPED_BY_STREAM = 0x20

STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEDOUT", -5: "ENOTFOUND", -6: "EBUSY"}

# every function the header declares
EXPORTED_SYMBOLS = (
    "talp_gpu_create", "talp_gpu_destroy", "talp_gpu_ingest_events", "talp_gpu_region_metrics",
    "talp_gpu_region_metrics_batch", "talp_gpu_region_metrics_device", "talp_gpu_metrics_combine",
    "talp_gpu_concurrency", "talp_gpu_scalability", "talp_gpu_ingest_raw", "talp_gpu_raw_held",
    "talp_gpu_unit_sums", "talp_gpu_thread_metrics", "talp_gpu_thread_metrics_device",
    "talp_gpu_thread_metrics_combine",
    "talp_gpu_reset", "talp_gpu_memory", "talp_gpu_profile", "talp_gpu_profile_read", "talp_gpu_reduce_noalloc",
    "talp_gpu_plan_create", "talp_gpu_plan_launch", "talp_gpu_plan_metrics", "talp_gpu_plan_info",
    "talp_gpu_plan_destroy", "talp_gpu_server_create", "talp_gpu_server_open_job", "talp_gpu_server_submit", "talp_gpu_server_submit_raw",
    "talp_gpu_server_query", "talp_gpu_server_query_threads", "talp_gpu_server_drain", "talp_gpu_server_close_job", "talp_gpu_server_info",
    "talp_gpu_server_destroy", "talp_gpu_last_error",
)
TALP_GPU_PLAN_AUTOTUNE = 0x1
TALP_GPU_NOALLOC_MAX_UNITS = 8192
TALP_GPU_CONC_LEVELS = 8


class TalpGpuError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class talp_gpu_trace_batch(ctypes.Structure):
    _fields_ = [
        ("trace_id", ctypes.c_uint64),
        ("n_ranks", ctypes.c_uint32),
        ("n_regions", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("devices_per_rank", ctypes.c_void_p),
        ("region_window", ctypes.c_void_p),
        ("host_se", ctypes.c_void_p),
        ("host_state", ctypes.c_void_p),
        ("host_off", ctypes.c_void_p),
        ("dev_se", ctypes.c_void_p),
        ("dev_tag", ctypes.c_void_p),
        ("dev_off", ctypes.c_void_p),
    ]


INT_FIELDS = ("elapsed_ns", "sum_useful", "sum_offload", "sum_mpi", "max_useful_offload",
              "sum_kernel", "max_kernel", "max_busy", "sum_mem", "sum_idle", "sum_hidden_mem")
RATIO_FIELDS = ("host_pe", "host_mpi_pe", "host_mpi_lb", "host_mpi_ce", "host_oe",
                "dev_pe", "dev_lb", "dev_ce", "dev_oe")


class talp_gpu_profile_stats(ctypes.Structure):
    _fields_ = [("sweep_launches", ctypes.c_uint64), ("sweep_records", ctypes.c_uint64),
                ("sweep_ms", ctypes.c_double), ("kernel_launches", ctypes.c_uint64),
                ("sort_launches", ctypes.c_uint64), ("sort_ms", ctypes.c_double)]


class talp_gpu_plan_stats(ctypes.Structure):
    _fields_ = [("n_metrics", ctypes.c_uint64), ("records", ctypes.c_uint64), ("segments", ctypes.c_uint64),
                ("kernels_per_launch", ctypes.c_uint32), ("sweep_items", ctypes.c_uint32),
                ("sweep_warps", ctypes.c_uint32), ("sweep_stages", ctypes.c_uint32),
                ("tiles_per_warp", ctypes.c_uint32), ("sweep_grid", ctypes.c_uint32), ("slices_per_warp", ctypes.c_uint32)]


class talp_gpu_server_config(ctypes.Structure):
    _fields_ = [("max_jobs", ctypes.c_uint32), ("max_slice_records", ctypes.c_uint32),
                ("staging_slices", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class talp_gpu_server_stats(ctypes.Structure):
    _fields_ = [("slices_submitted", ctypes.c_uint64), ("slices_folded", ctypes.c_uint64),
                ("records_folded", ctypes.c_uint64), ("waves", ctypes.c_uint64), ("queries", ctypes.c_uint64),
                ("query_batches", ctypes.c_uint64), ("query_p50_ms", ctypes.c_double),
                ("query_p99_ms", ctypes.c_double), ("query_max_ms", ctypes.c_double),
                ("jobs_open", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class talp_gpu_raw_batch(ctypes.Structure):
    _fields_ = [
        ("trace_id", ctypes.c_uint64), ("n_ranks", ctypes.c_uint32), ("n_regions", ctypes.c_uint32),
        ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("devices_per_rank", ctypes.c_void_p),
        ("region_window", ctypes.c_void_p), ("host_se", ctypes.c_void_p), ("host_state", ctypes.c_void_p),
        ("host_off", ctypes.c_void_p), ("raw_se", ctypes.c_void_p), ("raw_tag", ctypes.c_void_p),
        ("raw_dev", ctypes.c_void_p), ("raw_off", ctypes.c_void_p), ("stream_mask", ctypes.c_void_p),
    ]


class talp_gpu_scaling(ctypes.Structure):
    _fields_ = [("trace_id", ctypes.c_uint64), ("region", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("n_ranks", ctypes.c_uint32), ("m_devices", ctypes.c_uint32), ("speedup", ctypes.c_double),
                ("host_comp_scal", ctypes.c_double), ("host_global_eff", ctypes.c_double),
                ("dev_comp_scal", ctypes.c_double), ("dev_global_eff", ctypes.c_double)]


THREAD_INT_FIELDS = ("elapsed_ns", "sum_useful", "sum_offload", "sum_busiest", "max_busiest")
THREAD_RATIO_FIELDS = ("pe", "mpi_pe", "mpi_lb", "mpi_ce", "thread_lb", "oe")


class talp_gpu_thread_tree(ctypes.Structure):
    _fields_ = ([("trace_id", ctypes.c_uint64), ("region", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                 ("n_procs", ctypes.c_uint32), ("n_threads", ctypes.c_uint32)]
                + [(f, ctypes.c_int64) for f in THREAD_INT_FIELDS]
                + [(f, ctypes.c_double) for f in THREAD_RATIO_FIELDS])


class talp_gpu_metrics(ctypes.Structure):
    _fields_ = ([("trace_id", ctypes.c_uint64), ("region", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                 ("n_ranks", ctypes.c_uint32), ("m_devices", ctypes.c_uint32)]
                + [(f, ctypes.c_int64) for f in INT_FIELDS]
                + [(f, ctypes.c_double) for f in RATIO_FIELDS])


def metrics_to_dict(m: talp_gpu_metrics) -> dict:
    d = {f: int(getattr(m, f)) for f in INT_FIELDS}
    d.update({f: float(getattr(m, f)) for f in RATIO_FIELDS})
    d.update(trace_id=int(m.trace_id), region=int(m.region), flags=int(m.flags), n_ranks=int(m.n_ranks),
             m_devices=int(m.m_devices))
    return d


def metrics_from_dict(d: dict) -> talp_gpu_metrics:
    m = talp_gpu_metrics()
    for f, _ in talp_gpu_metrics._fields_:
        setattr(m, f, d[f])
    return m


_lib = None


def load_library():
    """Load libtalp_gpu.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library missing: {LIB_PATH} (build it with `python -m paper_2603_26576_b300.build`)")
    lib = ctypes.CDLL(LIB_PATH)
    P, S = ctypes.c_void_p, ctypes.c_size_t
    I32, U32, U64 = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
    sig = {
        "talp_gpu_create": ([ctypes.POINTER(ctypes.c_void_p), I32, S], I32),
        "talp_gpu_destroy": ([P], I32),
        "talp_gpu_ingest_events": ([P, ctypes.POINTER(talp_gpu_trace_batch), S, P], I32),
        "talp_gpu_region_metrics": ([P, U64, U32, ctypes.POINTER(talp_gpu_metrics), P], I32),
        "talp_gpu_region_metrics_batch": ([P, P, S, U32, ctypes.POINTER(talp_gpu_metrics), P], I32),
        "talp_gpu_region_metrics_device": ([P, P, S, U32, P, P], I32),
        "talp_gpu_metrics_combine": ([P, ctypes.POINTER(talp_gpu_metrics), S, ctypes.POINTER(talp_gpu_metrics), P],
                                     I32),
        "talp_gpu_unit_sums": ([P, U64, U32, P, P, P], I32),
        "talp_gpu_thread_metrics": ([P, U64, U32, P, U32, ctypes.POINTER(talp_gpu_thread_tree), P], I32),
        "talp_gpu_thread_metrics_device": ([P, U64, U32, P, U32, P, P], I32),
        "talp_gpu_thread_metrics_combine": ([P, ctypes.POINTER(talp_gpu_thread_tree), S,
                                             ctypes.POINTER(talp_gpu_thread_tree), P], I32),
        "talp_gpu_concurrency": ([P, ctypes.POINTER(talp_gpu_trace_batch), U32, P, P], I32),
        "talp_gpu_scalability": ([P, ctypes.POINTER(talp_gpu_metrics), S, S, U32, ctypes.POINTER(talp_gpu_scaling),
                                  P], I32),
        "talp_gpu_ingest_raw": ([P, ctypes.POINTER(talp_gpu_raw_batch), S, P], I32),
        "talp_gpu_raw_held": ([P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)], I32),
        "talp_gpu_reset": ([P, U64], I32),
        "talp_gpu_memory": ([P, ctypes.POINTER(S), ctypes.POINTER(S)], I32),
        "talp_gpu_profile": ([P, I32], I32),
        "talp_gpu_profile_read": ([P, ctypes.POINTER(talp_gpu_profile_stats)], I32),
        "talp_gpu_reduce_noalloc": ([ctypes.POINTER(talp_gpu_trace_batch), ctypes.POINTER(talp_gpu_metrics), P], I32),
        "talp_gpu_plan_create": ([P, ctypes.POINTER(talp_gpu_trace_batch), S, U32, ctypes.POINTER(ctypes.c_void_p)],
                                 I32),
        "talp_gpu_plan_launch": ([P, P], I32),
        "talp_gpu_plan_metrics": ([P, ctypes.POINTER(talp_gpu_metrics), P], I32),
        "talp_gpu_plan_info": ([P, ctypes.POINTER(talp_gpu_plan_stats)], I32),
        "talp_gpu_plan_destroy": ([P], I32),
        "talp_gpu_server_create": ([P, ctypes.POINTER(talp_gpu_server_config), ctypes.POINTER(ctypes.c_void_p)],
                                   I32),
        "talp_gpu_server_open_job": ([P, U64, U32, P, U32, P], I32),
        "talp_gpu_server_submit": ([P, U64, ctypes.POINTER(talp_gpu_trace_batch)], I32),
        "talp_gpu_server_submit_raw": ([P, U64, ctypes.POINTER(talp_gpu_raw_batch)], I32),
        "talp_gpu_server_query": ([P, U64, U32, ctypes.POINTER(talp_gpu_metrics)], I32),
        "talp_gpu_server_query_threads": ([P, U64, U32, P, U32, ctypes.POINTER(talp_gpu_thread_tree)], I32),
        "talp_gpu_server_drain": ([P], I32),
        "talp_gpu_server_close_job": ([P, U64], I32),
        "talp_gpu_server_info": ([P, ctypes.POINTER(talp_gpu_server_stats)], I32),
        "talp_gpu_server_destroy": ([P], I32),
        "talp_gpu_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def talp_gpu_last_error() -> str:
    return load_library().talp_gpu_last_error().decode()


def _check(st):
    if st != 0:
        raise TalpGpuError(st, talp_gpu_last_error())


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def talp_gpu_create(device: int = 0, hbm_budget_bytes: int = 0):
    ctx = ctypes.c_void_p()
    _check(load_library().talp_gpu_create(ctypes.byref(ctx), device, hbm_budget_bytes))
    return ctx


def talp_gpu_destroy(ctx):
    _check(load_library().talp_gpu_destroy(ctx))


def talp_gpu_ingest_events(ctx, batches, stream=None):
    arr = (talp_gpu_trace_batch * len(batches))(*batches)
    _check(load_library().talp_gpu_ingest_events(ctx, arr, len(batches), _stream(stream)))


def talp_gpu_region_metrics(ctx, trace_id, region, stream=None, n_regions=None, check=True):
    """Metrics of one region (a talp_gpu_metrics) or, with
    region=TALP_GPU_ALL_REGIONS, a list over the n_regions regions."""
    k = n_regions if region == TALP_GPU_ALL_REGIONS else 1
    if k is None:
        raise ValueError("n_regions is needed with TALP_GPU_ALL_REGIONS")
    out = (talp_gpu_metrics * k)()
    st = load_library().talp_gpu_region_metrics(ctx, trace_id, region, out, _stream(stream))
    res = list(out) if region == TALP_GPU_ALL_REGIONS else out[0]
    if check:
        _check(st)
        return res
    return st, res


def talp_gpu_thread_metrics(ctx, trace_id, region, proc_off, stream=None, n_regions=None, check=True):
    """Host tree with threads of one region (a dict) or, with
    region=TALP_GPU_ALL_REGIONS, a list of dicts over the n_regions regions;
    proc_off (n_procs + 1 entries) groups the trace's host units into
    processes."""
    k = n_regions if region == TALP_GPU_ALL_REGIONS else 1
    if k is None:
        raise ValueError("n_regions is needed with TALP_GPU_ALL_REGIONS")
    po = np.ascontiguousarray(proc_off, dtype=np.uint32)
    if po.ndim != 1 or po.shape[0] < 1:
        raise ValueError("proc_off needs n_procs + 1 entries")
    out = (talp_gpu_thread_tree * k)()
    st = load_library().talp_gpu_thread_metrics(ctx, trace_id, region, po.ctypes.data_as(ctypes.c_void_p),
                                                po.shape[0] - 1, out, _stream(stream))
    res = [{f: (float(getattr(o, f)) if t is ctypes.c_double else int(getattr(o, f))) for f, t in o._fields_}
           for o in out]
    res = res if region == TALP_GPU_ALL_REGIONS else res[0]
    if check:
        _check(st)
        return res
    return st, res


def talp_gpu_thread_metrics_device(ctx, trace_id, region, proc_off, out_device_ptr, stream=None):
    """Stream-ordered thread tree into device memory (one talp_gpu_thread_tree
    per region at out_device_ptr)."""
    po = np.ascontiguousarray(proc_off, dtype=np.uint32)
    _check(load_library().talp_gpu_thread_metrics_device(ctx, trace_id, region, po.ctypes.data_as(ctypes.c_void_p),
                                                         po.shape[0] - 1, out_device_ptr, _stream(stream)))


def talp_gpu_thread_metrics_combine(ctx, parts, stream=None, check=True):
    """Thread-tree records (dicts as talp_gpu_thread_metrics returns) of one
    region on disjoint shards -> the whole trace's record (a dict)."""
    arr = (talp_gpu_thread_tree * max(1, len(parts)))()
    for k, p in enumerate(parts):
        for f, _ in talp_gpu_thread_tree._fields_:
            setattr(arr[k], f, p[f])
    out = talp_gpu_thread_tree()
    st = load_library().talp_gpu_thread_metrics_combine(ctx, arr, len(parts), ctypes.byref(out), _stream(stream))
    res = {f: (float(getattr(out, f)) if t is ctypes.c_double else int(getattr(out, f)))
           for f, t in out._fields_}
    if check:
        _check(st)
        return res
    return st, res


def thread_tree_from_bytes(buf) -> list:
    """talp_gpu_thread_tree records (as dicts) from their raw bytes."""
    n = len(buf) // ctypes.sizeof(talp_gpu_thread_tree)
    arr = (talp_gpu_thread_tree * n).from_buffer_copy(bytes(buf[: n * ctypes.sizeof(talp_gpu_thread_tree)]))
    return [{f: (float(getattr(o, f)) if t is ctypes.c_double else int(getattr(o, f))) for f, t in o._fields_}
            for o in arr]


def talp_gpu_region_metrics_batch(ctx, trace_ids, region, stream=None, check=True):
    ids = np.ascontiguousarray(trace_ids, dtype=np.uint64)
    out = (talp_gpu_metrics * len(ids))()
    st = load_library().talp_gpu_region_metrics_batch(ctx, ids.ctypes.data_as(ctypes.c_void_p), len(ids), region,
                                                      out, _stream(stream))
    if check:
        _check(st)
        return list(out)
    return st, list(out)


def talp_gpu_region_metrics_device(ctx, trace_ids, region, out_device_ptr, stream=None):
    ids = np.ascontiguousarray(trace_ids, dtype=np.uint64)
    _check(load_library().talp_gpu_region_metrics_device(ctx, ids.ctypes.data_as(ctypes.c_void_p), len(ids),
                                                         region, ctypes.c_void_p(out_device_ptr), _stream(stream)))


def talp_gpu_metrics_combine(ctx, parts, stream=None, check=True):
    """Metrics of a region of a trace from its shards' metrics (a list of
    talp_gpu_metrics or of dicts as metrics_to_dict returns)."""
    arr = (talp_gpu_metrics * len(parts))()
    for k, p in enumerate(parts):
        arr[k] = p if isinstance(p, talp_gpu_metrics) else metrics_from_dict(p)
    out = talp_gpu_metrics()
    st = load_library().talp_gpu_metrics_combine(ctx, arr, len(parts), ctypes.byref(out), _stream(stream))
    if check:
        _check(st)
        return out
    return st, out


def talp_gpu_concurrency(ctx, batch, region, stream=None, check=True):
    """int64[m, 2, TALP_GPU_CONC_LEVELS]: per device, time with at least k
    active records (all, then kernels only) in the region."""
    m = int(np.ctypeslib.as_array(ctypes.cast(batch.devices_per_rank, ctypes.POINTER(ctypes.c_uint32)),
                                  shape=(batch.n_ranks,)).sum())
    out = np.zeros((m, 2, TALP_GPU_CONC_LEVELS), np.int64)
    st = load_library().talp_gpu_concurrency(ctx, ctypes.byref(batch), region,
                                             out.ctypes.data_as(ctypes.c_void_p), _stream(stream))
    if check:
        _check(st)
        return out
    return st, out


def raw_batch_from_arrays(trace_id, devices_per_rank, region_window, host_se, host_state, host_off, raw_se,
                          raw_tag, raw_dev, raw_off, flags=0, stream_mask=None):
    """Build a talp_gpu_raw_batch (record arrays: all numpy host arrays, or
    all CUDA tensors; stream_mask: host [n_ranks][8] or None).  Returns
    (batch, keepalive)."""
    dpr = np.ascontiguousarray(devices_per_rank, dtype=np.uint32)
    win = np.ascontiguousarray(region_window, dtype=np.int64)
    hoff = np.ascontiguousarray(host_off, dtype=np.uint64)
    roff = np.ascontiguousarray(raw_off, dtype=np.uint64)
    keep = [dpr, win, hoff, roff]
    smask = None
    if stream_mask is not None:
        smask = np.ascontiguousarray(stream_mask, dtype=np.uint32).reshape(dpr.shape[0], 8)
        keep.append(smask)
    ptrs, dev_flags = [], set()
    for a, dt in ((host_se, np.int64), (host_state, np.uint8), (raw_se, np.int64), (raw_tag, np.uint8),
                  (raw_dev, np.uint8)):
        if not hasattr(a, "data_ptr"):
            a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        p, is_dev = _ptr(a)
        ptrs.append(p)
        dev_flags.add(is_dev)
    if len(dev_flags) != 1:
        raise ValueError("record arrays must be all host or all device")
    if dev_flags.pop():
        flags |= TALP_GPU_DEVICE_PTRS
    b = talp_gpu_raw_batch()
    b.trace_id, b.n_ranks, b.n_regions, b.flags, b.reserved = int(trace_id), int(dpr.shape[0]), int(win.shape[0]), \
        int(flags), 0
    b.devices_per_rank, b.region_window, b.host_off, b.raw_off = dpr.ctypes.data, win.ctypes.data, hoff.ctypes.data, \
        roff.ctypes.data
    b.host_se, b.host_state, b.raw_se, b.raw_tag, b.raw_dev = ptrs
    b.stream_mask = smask.ctypes.data if smask is not None else None
    return b, keep


def talp_gpu_ingest_raw(ctx, batches, stream=None):
    arr = (talp_gpu_raw_batch * len(batches))(*batches)
    _check(load_library().talp_gpu_ingest_raw(ctx, arr, len(batches), _stream(stream)))


def talp_gpu_raw_held(ctx, trace_id):
    out = ctypes.c_uint64(0)
    _check(load_library().talp_gpu_raw_held(ctx, int(trace_id), ctypes.byref(out)))
    return int(out.value)


def talp_gpu_scalability(ctx, runs, ref=0, weak=False, stream=None, check=True):
    """Scaling factors of region metrics `runs` (structs or dicts) against
    runs[ref]; a list of dicts."""
    arr = (talp_gpu_metrics * len(runs))()
    for k, p in enumerate(runs):
        arr[k] = p if isinstance(p, talp_gpu_metrics) else metrics_from_dict(p)
    out = (talp_gpu_scaling * max(1, len(runs)))()
    st = load_library().talp_gpu_scalability(ctx, arr, len(runs), ref, 1 if weak else 0, out, _stream(stream))
    res = [{f: (float(getattr(o, f)) if t is ctypes.c_double else int(getattr(o, f))) for f, t in o._fields_}
           for o in list(out)[:len(runs)]]
    if check:
        _check(st)
        return res
    return st, res


def talp_gpu_unit_sums(ctx, trace_id, region, n_ranks, m_devices, stream=None):
    h = np.zeros((n_ranks, 3), np.int64)
    d = np.zeros((m_devices, 3), np.int64)
    _check(load_library().talp_gpu_unit_sums(ctx, trace_id, region, h.ctypes.data_as(ctypes.c_void_p),
                                             d.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return h, d


def talp_gpu_reset(ctx, trace_id=TALP_GPU_ALL):
    _check(load_library().talp_gpu_reset(ctx, trace_id))


def talp_gpu_memory(ctx):
    held, budget = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load_library().talp_gpu_memory(ctx, ctypes.byref(held), ctypes.byref(budget)))
    return held.value, budget.value


def talp_gpu_profile(ctx, enable=True):
    _check(load_library().talp_gpu_profile(ctx, 1 if enable else 0))


def talp_gpu_profile_read(ctx) -> dict:
    st = talp_gpu_profile_stats()
    _check(load_library().talp_gpu_profile_read(ctx, ctypes.byref(st)))
    return dict(sweep_launches=int(st.sweep_launches), sweep_records=int(st.sweep_records),
                sweep_ms=float(st.sweep_ms), kernel_launches=int(st.kernel_launches),
                sort_launches=int(st.sort_launches), sort_ms=float(st.sort_ms))


def talp_gpu_plan_create(ctx, batches, plan_flags=0):
    arr = (talp_gpu_trace_batch * len(batches))(*batches)
    plan = ctypes.c_void_p()
    _check(load_library().talp_gpu_plan_create(ctx, arr, len(batches), plan_flags, ctypes.byref(plan)))
    return plan


def talp_gpu_plan_launch(plan, stream=None):
    _check(load_library().talp_gpu_plan_launch(plan, _stream(stream)))


def talp_gpu_plan_info(plan) -> dict:
    st = talp_gpu_plan_stats()
    _check(load_library().talp_gpu_plan_info(plan, ctypes.byref(st)))
    return {f: int(getattr(st, f)) for f, _ in talp_gpu_plan_stats._fields_}


def talp_gpu_plan_metrics(plan, stream=None, check=True):
    n = talp_gpu_plan_info(plan)["n_metrics"]
    out = (talp_gpu_metrics * max(1, n))()
    st = load_library().talp_gpu_plan_metrics(plan, out, _stream(stream))
    res = list(out)[:n]
    if check:
        _check(st)
        return res
    return st, res


def talp_gpu_plan_destroy(plan):
    _check(load_library().talp_gpu_plan_destroy(plan))


def talp_gpu_reduce_noalloc(batch, stream=None, check=True):
    """Metrics of every region of one trace with no device allocation (the
    records must be device memory in start order).  Returns a list of
    talp_gpu_metrics, one per region."""
    out = (talp_gpu_metrics * max(1, batch.n_regions))()
    st = load_library().talp_gpu_reduce_noalloc(ctypes.byref(batch), out, _stream(stream))
    res = list(out)[: batch.n_regions]
    if check:
        _check(st)
        return res
    return st, res


def talp_gpu_server_create(ctx, max_jobs=0, max_slice_records=0, staging_slices=0):
    cfg = talp_gpu_server_config(max_jobs, max_slice_records, staging_slices, 0)
    srv = ctypes.c_void_p()
    _check(load_library().talp_gpu_server_create(ctx, ctypes.byref(cfg), ctypes.byref(srv)))
    return srv


def talp_gpu_server_open_job(srv, job_id, devices_per_rank, region_window, check=True):
    dpr = np.ascontiguousarray(devices_per_rank, dtype=np.uint32)
    win = np.ascontiguousarray(region_window, dtype=np.int64)
    st = load_library().talp_gpu_server_open_job(srv, int(job_id), int(dpr.shape[0]),
                                                 dpr.ctypes.data_as(ctypes.c_void_p), int(win.shape[0]),
                                                 win.ctypes.data_as(ctypes.c_void_p))
    if check:
        _check(st)
    return st


def talp_gpu_server_submit(srv, job_id, batch, check=True):
    st = load_library().talp_gpu_server_submit(srv, int(job_id), ctypes.byref(batch))
    if check:
        _check(st)
    return st


def talp_gpu_server_submit_raw(srv, job_id, batch, check=True):
    st = load_library().talp_gpu_server_submit_raw(srv, int(job_id), ctypes.byref(batch))
    if check:
        _check(st)
    return st


def talp_gpu_server_query(srv, job_id, region, n_regions=None, check=True):
    k = n_regions if region == TALP_GPU_ALL_REGIONS else 1
    if k is None:
        raise ValueError("n_regions is needed with TALP_GPU_ALL_REGIONS")
    out = (talp_gpu_metrics * k)()
    st = load_library().talp_gpu_server_query(srv, int(job_id), region, out)
    res = list(out) if region == TALP_GPU_ALL_REGIONS else out[0]
    if check:
        _check(st)
        return res
    return st, res


def talp_gpu_server_query_threads(srv, job_id, region, proc_off, n_regions=None, check=True):
    """Host tree with threads of a served job (a dict, or a list of dicts with
    TALP_GPU_ALL_REGIONS)."""
    k = n_regions if region == TALP_GPU_ALL_REGIONS else 1
    if k is None:
        raise ValueError("n_regions is needed with TALP_GPU_ALL_REGIONS")
    po = np.ascontiguousarray(proc_off, dtype=np.uint32)
    if po.ndim != 1 or po.shape[0] < 1:
        raise ValueError("proc_off needs n_procs + 1 entries")
    out = (talp_gpu_thread_tree * k)()
    st = load_library().talp_gpu_server_query_threads(srv, int(job_id), region, po.ctypes.data_as(ctypes.c_void_p),
                                                      po.shape[0] - 1, out)
    res = [{f: (float(getattr(o, f)) if t is ctypes.c_double else int(getattr(o, f))) for f, t in o._fields_}
           for o in out]
    res = res if region == TALP_GPU_ALL_REGIONS else res[0]
    if check:
        _check(st)
        return res
    return st, res


def talp_gpu_server_drain(srv):
    _check(load_library().talp_gpu_server_drain(srv))


def talp_gpu_server_close_job(srv, job_id):
    _check(load_library().talp_gpu_server_close_job(srv, int(job_id)))


def talp_gpu_server_info(srv) -> dict:
    st = talp_gpu_server_stats()
    _check(load_library().talp_gpu_server_info(srv, ctypes.byref(st)))
    return {f: (float(getattr(st, f)) if t is ctypes.c_double else int(getattr(st, f)))
            for f, t in talp_gpu_server_stats._fields_ if f != "reserved"}


def talp_gpu_server_destroy(srv):
    _check(load_library().talp_gpu_server_destroy(srv))


# ----------------------------------------------------------------- marshalling


def _ptr(a):
    """(address, is_device) of a numpy array or a torch tensor."""
    if a is None:
        return None, False
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), bool(a.is_cuda)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("arrays must be C-contiguous")
    return a.ctypes.data, False


def batch_from_arrays(trace_id, devices_per_rank, region_window, host_se, host_state, host_off,
                      dev_se, dev_tag, dev_off, flags=0):
    """Build a talp_gpu_trace_batch.  Header arrays (devices_per_rank,
    region_window, offsets) are host numpy arrays; record arrays are numpy
    arrays (host) or CUDA tensors (device; TALP_GPU_DEVICE_PTRS is then set).
    Returns (batch, keepalive): keep `keepalive` referenced until the ingest
    call's stream has passed it."""
    dpr = np.ascontiguousarray(devices_per_rank, dtype=np.uint32)
    win = np.ascontiguousarray(region_window, dtype=np.int64)
    hoff = np.ascontiguousarray(host_off, dtype=np.uint64)
    doff = np.ascontiguousarray(dev_off, dtype=np.uint64)
    keep = [dpr, win, hoff, doff]
    ptrs = []
    dev_flags = set()
    for a, dt in ((host_se, np.int64), (host_state, np.uint8), (dev_se, np.int64), (dev_tag, np.uint8)):
        if not hasattr(a, "data_ptr"):
            a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        p, is_dev = _ptr(a)
        ptrs.append(p)
        dev_flags.add(is_dev)
    if len(dev_flags) != 1:
        raise ValueError("record arrays must be all host or all device")
    if dev_flags.pop():
        flags |= TALP_GPU_DEVICE_PTRS
    b = talp_gpu_trace_batch()
    b.trace_id = int(trace_id)
    b.n_ranks = int(dpr.shape[0])
    b.n_regions = int(win.shape[0])
    b.flags = int(flags)
    b.reserved = 0
    b.devices_per_rank = dpr.ctypes.data
    b.region_window = win.ctypes.data
    b.host_se, b.host_state, b.dev_se, b.dev_tag = ptrs
    b.host_off = hoff.ctypes.data
    b.dev_off = doff.ctypes.data
    return b, keep


class Context:
    """Owning wrapper of a talp_gpu_ctx."""

    def __init__(self, device=0, hbm_budget_bytes=0):
        self.ctx = talp_gpu_create(device, hbm_budget_bytes)
        self._keep = []
        self._shapes = {}

    def close(self):
        if self.ctx is not None:
            talp_gpu_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ingest(self, traces, flags=0, stream=None, arrays=None):
        """Ingest trace objects (attributes as produced by tracegen).  With
        `arrays`, a parallel list of dicts overriding the record arrays (e.g.
        CUDA tensors) is used."""
        batches, keep = [], []
        for k, t in enumerate(traces):
            rec = dict(host_se=t.host_se, host_state=t.host_state, dev_se=t.dev_se, dev_tag=t.dev_tag)
            if arrays is not None:
                rec.update(arrays[k])
            b, kp = batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, rec["host_se"],
                                      rec["host_state"], t.host_off, rec["dev_se"], rec["dev_tag"], t.dev_off,
                                      flags)
            batches.append(b)
            keep.append(kp)
            self._shapes[int(t.trace_id)] = (int(t.n_ranks), int(np.asarray(t.devices_per_rank).sum()),
                                             int(np.asarray(t.region_window).shape[0]))
        talp_gpu_ingest_events(self.ctx, batches, stream)
        self._keep = keep
        return batches

    def metrics(self, trace_id, region=TALP_GPU_ALL_REGIONS, stream=None, check=True):
        R = self._shapes[int(trace_id)][2]
        r = talp_gpu_region_metrics(self.ctx, trace_id, region, stream, n_regions=R, check=check)
        if not check:
            st, r = r
            conv = [metrics_to_dict(x) for x in r] if isinstance(r, list) else metrics_to_dict(r)
            return st, conv
        return [metrics_to_dict(x) for x in r] if isinstance(r, list) else metrics_to_dict(r)

    def metrics_batch(self, trace_ids, region, stream=None):
        return [metrics_to_dict(x) for x in talp_gpu_region_metrics_batch(self.ctx, trace_ids, region, stream)]

    def thread_metrics(self, trace_id, proc_off, region=TALP_GPU_ALL_REGIONS, stream=None, check=True):
        """Host tree with threads: the trace's host units are threads,
        grouped into processes by proc_off."""
        R = self._shapes[int(trace_id)][2]
        return talp_gpu_thread_metrics(self.ctx, trace_id, region, proc_off, stream, n_regions=R, check=check)

    def unit_sums(self, trace_id, region, stream=None):
        n, m, _ = self._shapes[int(trace_id)]
        return talp_gpu_unit_sums(self.ctx, trace_id, region, n, m, stream)

    def reset(self, trace_id=TALP_GPU_ALL):
        talp_gpu_reset(self.ctx, trace_id)
        if trace_id == TALP_GPU_ALL:
            self._shapes.clear()
        else:
            self._shapes.pop(int(trace_id), None)

    def memory(self):
        return talp_gpu_memory(self.ctx)

    def ingest_raw(self, raws, flags=0, stream=None, arrays=None):
        """Ingest raw activity records (objects with .trace and raw_se /
        raw_tag / raw_dev / raw_off as tracegen.to_raw makes, and a
        stream_mask attribute for TALP_GPU_HOLD_BACK); `flags` is one
        word for all or a list with one per trace; `arrays` may hold CUDA
        tensors for the five record arrays of each."""
        batches, keep = [], []
        fl = list(flags) if isinstance(flags, (list, tuple)) else [flags] * len(raws)
        for k, r in enumerate(raws):
            t = r.trace
            rec = dict(host_se=t.host_se, host_state=t.host_state, raw_se=r.raw_se, raw_tag=r.raw_tag,
                       raw_dev=r.raw_dev)
            if arrays is not None:
                rec.update(arrays[k])
            b, kp = raw_batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, rec["host_se"],
                                          rec["host_state"], t.host_off, rec["raw_se"], rec["raw_tag"],
                                          rec["raw_dev"], r.raw_off, fl[k], getattr(r, "stream_mask", None))
            batches.append(b)
            keep.append(kp)
            self._shapes[int(t.trace_id)] = (int(t.n_ranks), int(np.asarray(t.devices_per_rank).sum()),
                                             int(np.asarray(t.region_window).shape[0]))
        talp_gpu_ingest_raw(self.ctx, batches, stream)
        self._keep = keep

    def raw_held(self, trace_id):
        """Raw records of the trace held back and not folded yet."""
        return talp_gpu_raw_held(self.ctx, trace_id)

    def concurrency(self, t, region, arrays=None, stream=None, check=True):
        """Concurrency profile of trace `t` (records in start order) in one
        region; `arrays` may hold CUDA tensors for dev_se / dev_tag."""
        rec = dict(host_se=t.host_se, host_state=t.host_state, dev_se=t.dev_se, dev_tag=t.dev_tag)
        if arrays is not None:
            rec.update(arrays)
        b, keep = batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, rec["host_se"],
                                    rec["host_state"], t.host_off, rec["dev_se"], rec["dev_tag"], t.dev_off)
        return talp_gpu_concurrency(self.ctx, b, region, stream, check)

    def plan(self, traces, arrays, flags=TALP_GPU_SORTED_BY_START, plan_flags=0):
        """A batched plan over traces whose records are the CUDA tensors in
        `arrays` (one dict per trace: host_se, host_state, dev_se, dev_tag)."""
        batches, keep = [], []
        for t, a in zip(traces, arrays):
            b, kp = batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, a["host_se"],
                                      a["host_state"], t.host_off, a["dev_se"], a["dev_tag"], t.dev_off, flags)
            batches.append(b)
            keep.append(kp)
            self._shapes[int(t.trace_id)] = (int(t.n_ranks), int(np.asarray(t.devices_per_rank).sum()),
                                             int(np.asarray(t.region_window).shape[0]))
        return Plan(talp_gpu_plan_create(self.ctx, batches, plan_flags), keep, self)


class Plan:
    """Owning wrapper of a talp_gpu_plan (the batched form)."""

    def __init__(self, handle, keep, context=None):
        self.handle = handle
        self._keep = keep
        self.context = context   # destroyed after the plan

    def launch(self, stream=None):
        talp_gpu_plan_launch(self.handle, stream)

    def metrics(self, stream=None, check=True):
        r = talp_gpu_plan_metrics(self.handle, stream, check)
        if check:
            return [metrics_to_dict(x) for x in r]
        st, r = r
        return st, [metrics_to_dict(x) for x in r]

    def info(self):
        return talp_gpu_plan_info(self.handle)

    def close(self):
        if self.handle is not None:
            talp_gpu_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owning wrapper of a talp_gpu_server (the served form) on a Context.
    submit/query release the GIL inside the library, so client threads run
    concurrently."""

    def __init__(self, context, max_jobs=0, max_slice_records=0, staging_slices=0):
        self.context = context
        self.handle = talp_gpu_server_create(context.ctx, max_jobs, max_slice_records, staging_slices)
        self._R = {}

    def open_job(self, job_id, devices_per_rank, region_window, check=True):
        st = talp_gpu_server_open_job(self.handle, job_id, devices_per_rank, region_window, check)
        if st == 0:
            self._R[int(job_id)] = int(np.asarray(region_window).shape[0])
        return st

    def submit(self, job_id, host_se, host_state, host_off, dev_se, dev_tag, dev_off, sorted_by_start=True,
               check=True):
        """Queue one time slice (host numpy arrays, copied during the call)."""
        b, keep = batch_from_arrays(job_id, np.zeros(0, np.uint32), np.zeros((0, 0, 2), np.int64), host_se,
                                    host_state, host_off, dev_se, dev_tag, dev_off,
                                    TALP_GPU_SORTED_BY_START if sorted_by_start else 0)
        st = talp_gpu_server_submit(self.handle, job_id, b, check)
        del keep
        return st

    def submit_raw(self, job_id, host_se, host_state, host_off, raw_se, raw_tag, raw_dev, raw_off,
                   stream_mask=None, hold_back=True, check=True):
        """Queue one raw activity buffer (host numpy arrays, copied during the
        call); with hold_back, records a later buffer may precede are held
        back (stream_mask declares each device's streams)."""
        b, keep = raw_batch_from_arrays(job_id, np.zeros(0, np.uint32), np.zeros((0, 0, 2), np.int64), host_se,
                                        host_state, host_off, raw_se, raw_tag, raw_dev, raw_off,
                                        TALP_GPU_HOLD_BACK if hold_back else 0, None)
        sm = None
        if stream_mask is not None:
            sm = np.ascontiguousarray(stream_mask, dtype=np.uint32)
            b.stream_mask = sm.ctypes.data
        st = talp_gpu_server_submit_raw(self.handle, job_id, b, check)
        del keep, sm
        return st

    def query(self, job_id, region=TALP_GPU_ALL_REGIONS, check=True):
        r = talp_gpu_server_query(self.handle, job_id, region, self._R[int(job_id)], check)
        if not check:
            st, r = r
            return st, ([metrics_to_dict(x) for x in r] if isinstance(r, list) else metrics_to_dict(r))
        return [metrics_to_dict(x) for x in r] if isinstance(r, list) else metrics_to_dict(r)

    def query_threads(self, job_id, proc_off, region=TALP_GPU_ALL_REGIONS, check=True):
        return talp_gpu_server_query_threads(self.handle, job_id, region, proc_off, self._R[int(job_id)], check)

    def drain(self):
        talp_gpu_server_drain(self.handle)

    def close_job(self, job_id):
        talp_gpu_server_close_job(self.handle, job_id)
        self._R.pop(int(job_id), None)

    def stats(self):
        return talp_gpu_server_info(self.handle)

    def close(self):
        if self.handle is not None:
            talp_gpu_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
