"""Helpers for the GPU parity tests: contexts with a chosen sweep shape, and
element-by-element comparison against the oracle."""
import contextlib
import os
import struct

import numpy as np

import oracle
from oracle import INT_FIELDS, RATIO_FIELDS

# The GPU path is bit-exact by construction (exact int64 sums, the same FP64
# expression order, round to nearest, no contraction); the tolerance the
# requirement states is 1e-15 relative, the tests demand equality of bits.
REL_TOL = 0.0


def bits(x: float) -> int:
    return struct.unpack("<q", struct.pack("<d", x))[0]


def assert_metrics_equal(gpu: dict, orc: dict, tag=""):
    for k in INT_FIELDS:
        assert gpu[k] == orc[k], (tag, k, gpu[k], orc[k])
    for k in RATIO_FIELDS:
        assert bits(gpu[k]) == bits(orc[k]), (tag, k, repr(gpu[k]), repr(orc[k]))
    assert (gpu["flags"] & 0x7) == orc["flags"], (tag, "flags", gpu["flags"], orc["flags"])
    assert gpu["n_ranks"] == orc["n_ranks"] and gpu["m_devices"] == orc["m_devices"], tag


def assert_trace_equal(ctx, t, tag="", sums=True):
    res = ctx.metrics(t.trace_id)
    for r in range(t.n_regions):
        orc = oracle.region_metrics(t, r)
        assert_metrics_equal(res[r], orc, (tag, t.trace_id, r))
        if sums:
            h, d = ctx.unit_sums(t.trace_id, r)
            np.testing.assert_array_equal(h, oracle.host_sums(t, r), err_msg=str((tag, "host", r)))
            np.testing.assert_array_equal(d, oracle.device_unions(t, r), err_msg=str((tag, "dev", r)))


@contextlib.contextmanager
def env(**kv):
    old = {k: os.environ.get(k) for k in kv}
    try:
        for k, v in kv.items():
            os.environ[k] = str(v)
        yield
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def make_ctx(shape=None, tiles_per_warp=None, budget=0):
    import paper_2603_26576_b300 as P
    kv = {}
    if shape is not None:
        kv["TALP_GPU_SWEEP_SHAPE"] = shape
    if tiles_per_warp is not None:
        kv["TALP_GPU_TILES_PER_WARP"] = tiles_per_warp
    with env(**kv):
        return P.Context(0, budget)
