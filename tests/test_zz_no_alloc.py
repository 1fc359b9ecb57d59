"""The no-allocation entry point (talp_gpu_reduce_noalloc) against the regular
entry points, through the C ABI.

It is for callers that must not allocate device memory, e.g. a monitoring
hook inside the measured application whose allocator owns the GPU's memory.
Its results must equal those of a context's ingest + region_metrics bit for
bit (the tolerance of every parity test here), on two calls in a row with
different traces, since the calls share one scratch array.  This file is
named to be collected last.
"""
import numpy as np
import pytest

import tracegen as tg
from gpu_common import assert_metrics_equal

pytestmark = pytest.mark.gpu


def _device_batch(t):
    import torch
    import paper_2603_26576_b300 as P
    arrs = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
            for a in (t.host_se, t.host_state, t.dev_se, t.dev_tag)]
    b, keep = P.batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, arrs[0], arrs[1], t.host_off,
                                  arrs[2], arrs[3], t.dev_off, P.TALP_GPU_SORTED_BY_START)
    return b, keep + arrs


def _regular(t):
    import paper_2603_26576_b300 as P
    with P.Context(0) as c:
        c.ingest([t], flags=P.TALP_GPU_SORTED_BY_START)
        return c.metrics(t.trace_id)


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    import paper_2603_26576_b300 as P
    torch.cuda.init()
    traces = [
        tg.random_trace(21, trace_id=1, n_ranks=4, devices_per_rank=[1, 2, 0, 3], dev_events=[4000, 10, 2500, 0, 7000, 333],
                        host_events=[3000, 1, 0, 2222], n_regions=5),
        tg.single_trace_small(scale=0.3, trace_id=2),
    ]
    want = [_regular(t) for t in traces]
    torch.cuda.synchronize()
    free_before = None
    for call, (t, w) in enumerate(zip(traces, want)):
        b, keep = _device_batch(t)
        torch.cuda.synchronize()
        if call == 1:
            free_before = torch.cuda.mem_get_info()[0]
        got = [P.metrics_to_dict(x) for x in P.talp_gpu_reduce_noalloc(b)]
        assert len(got) == t.n_regions
        for r in range(t.n_regions):
            assert_metrics_equal(got[r], w[r], ("noalloc", call, r))
            for k in ("sum_kernel", "sum_mem", "elapsed_ns", "dev_pe", "host_pe"):
                assert got[r][k] == w[r][k]
    # the second call allocated no device memory
    assert torch.cuda.mem_get_info()[0] == free_before


def test_noalloc_rejects_sizes_beyond_the_limit():
    import paper_2603_26576_b300 as P
    n = P.TALP_GPU_NOALLOC_MAX_UNITS + 1
    dpr = np.zeros(n, np.uint32)
    win = np.zeros((1, n, 2), np.int64)
    empty_se = np.zeros((0, 2), np.int64)
    b, keep = P.batch_from_arrays(9, dpr, win, empty_se, np.zeros(0, np.uint8), np.zeros(n + 1, np.uint64),
                                  empty_se, np.zeros(0, np.uint8), np.zeros(1, np.uint64),
                                  P.TALP_GPU_SORTED_BY_START | P.TALP_GPU_DEVICE_PTRS)
    with pytest.raises(P.TalpGpuError) as ei:
        P.talp_gpu_reduce_noalloc(b)
    assert ei.value.status == -1
    assert "TALP_GPU_NOALLOC_MAX_UNITS" in str(ei.value)
