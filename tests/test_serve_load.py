"""The native client load of the serving workload (tracegen/serve_load), on
the CPU: fake submit and query entry points stand in for the library's and
record what the driver's threads hand them."""
import ctypes
import threading

import numpy as np
import pytest

import paper_2603_26576_b300 as P
from tracegen import serve_load

SUBMIT = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p)
EINVAL = -1  # talp_gpu_status TALP_GPU_EINVAL
QUERY = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p)


def _jobs(n_jobs=3, n_slices=2):
    """Tiny jobs of 2 ranks x 1 device: slice i holds host and device records
    with timestamps that tell job, slice and record apart."""
    keep, jobs, base = [], [], {}
    for j in range(n_jobs):
        arr = (P.talp_gpu_trace_batch * n_slices)()
        for i in range(n_slices):
            nh, nd = 2 + i, 3 + j
            hse = (np.arange(2 * nh, dtype=np.int64).reshape(nh, 2) + 1000 * j + 100 * i)
            dse = (np.arange(2 * nd, dtype=np.int64).reshape(nd, 2) + 1000 * j + 100 * i + 50)
            hoff = np.array([0, 1, nh], np.uint64)
            doff = np.array([0, nd - 1, nd], np.uint64)
            b, kp = P.batch_from_arrays(j, np.zeros(0, np.uint32), np.zeros((0, 0, 2), np.int64), hse,
                                        np.zeros(nh, np.uint8), hoff, dse, np.zeros(nd, np.uint8), doff,
                                        P.TALP_GPU_SORTED_BY_START)
            arr[i] = b
            keep.append(kp)
            base[(j, i)] = (hse.copy(), dse.copy())
        keep.append(arr)
        jobs.append(dict(job_id=j, n_ranks=2, n_devices=2, n_slices=n_slices, n_regions=3, span=10_000,
                         slices=ctypes.addressof(arr)))
    return jobs, keep, base


def test_slices_cycle_with_shift_and_queries_run():
    jobs, keep, base = _jobs()
    got = {}
    lock = threading.Lock()

    def fake_submit(srv, job_id, p):
        b = ctypes.cast(p, ctypes.POINTER(P.talp_gpu_trace_batch)).contents
        hoff = np.ctypeslib.as_array(ctypes.cast(b.host_off, ctypes.POINTER(ctypes.c_uint64)), (3,))
        doff = np.ctypeslib.as_array(ctypes.cast(b.dev_off, ctypes.POINTER(ctypes.c_uint64)), (3,))
        nh, nd = int(hoff[2]), int(doff[2])
        hse = np.ctypeslib.as_array(ctypes.cast(b.host_se, ctypes.POINTER(ctypes.c_int64)), (nh, 2)).copy()
        dse = np.ctypeslib.as_array(ctypes.cast(b.dev_se, ctypes.POINTER(ctypes.c_int64)), (nd, 2)).copy()
        with lock:
            got.setdefault(int(job_id), []).append((hse, dse, int(b.flags)))
        return 0

    nq = [0]

    def fake_query(srv, job_id, region, out):
        assert region == P.TALP_GPU_ALL_REGIONS
        with lock:
            nq[0] += 1
        return 0

    fs, fq = SUBMIT(fake_submit), QUERY(fake_query)
    addr = lambda f: ctypes.cast(f, ctypes.c_void_p).value  # noqa: E731
    next_q = [0, 1, 0]   # job 1 starts at its second slice
    r = serve_load.run(0x1234, addr(fs), addr(fq), jobs, next_q, rate=400.0, query_s=0.005, seconds=0.4,
                       n_sub=2, n_q=2)
    assert r["errors"] == 0 and r["first_error"] == 0
    assert r["slices"] == sum(len(v) for v in got.values()) > 10
    assert r["queries"] == nq[0] == len(r["lat"]) > 0
    assert all(x >= 0.0 for x in r["lat"])
    assert r["records"] == sum(h.shape[0] + d.shape[0] for v in got.values() for h, d, _ in v)
    start = {0: 0, 1: 1, 2: 0}
    for j, seq in got.items():
        # each job's slices in submission order: q, q + 1, ... with the shift of their cycle
        assert next_q[j] == start[j] + len(seq)
        for k, (h, d, flags) in enumerate(seq):
            q = start[j] + k
            hb, db = base[(j, q % 2)]
            shift = (q // 2) * 10_000
            np.testing.assert_array_equal(h, hb + shift)
            np.testing.assert_array_equal(d, db + shift)
            assert flags == P.TALP_GPU_SORTED_BY_START
    del keep


def test_failed_calls_are_counted_and_reported():
    jobs, keep, _ = _jobs(n_jobs=2)

    def ok_submit(srv, job_id, p):
        return 0

    def bad_query(srv, job_id, region, out):
        return EINVAL

    fs, fq = SUBMIT(ok_submit), QUERY(bad_query)
    addr = lambda f: ctypes.cast(f, ctypes.c_void_p).value  # noqa: E731
    r = serve_load.run(1, addr(fs), addr(fq), jobs, [0, 0], rate=200.0, query_s=0.01, seconds=0.2, n_sub=1, n_q=2)
    assert r["errors"] >= 1 and r["first_error"] == EINVAL
    del keep


def test_bad_arguments():
    jobs, keep, _ = _jobs(n_jobs=1)
    with pytest.raises(ValueError):
        serve_load.run(1, 0, 0, jobs, [0], rate=100.0, query_s=0.01, seconds=0.1)
    del keep
