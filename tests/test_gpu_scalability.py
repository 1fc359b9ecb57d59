"""Scalability across runs on the GPU: from the GPU's own region metrics of
several runs, the scaling factors equal the oracle's bit for bit."""
import struct

import pytest

import oracle
import tracegen as tg
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu

FIELDS = ("speedup", "host_comp_scal", "host_global_eff", "dev_comp_scal", "dev_global_eff")


def bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def test_scalability_matches_oracle():
    import paper_2603_26576_b300 as P
    c = make_ctx()
    shapes = [(1, 1), (2, 2), (4, 2), (8, 3), (16, 1)]
    traces = [tg.random_trace(90 + k, trace_id=k, n_ranks=n, devices_per_rank=g, dev_events=600, host_events=400,
                              n_regions=3) for k, (n, g) in enumerate(shapes)]
    c.ingest(traces)
    for region in range(3):
        gpu_runs = [c.metrics(t.trace_id, region) for t in traces]
        orc_runs = [oracle.region_metrics(t, region) for t in traces]
        for ref in (0, 3):
            for weak in (False, True):
                got = P.talp_gpu_scalability(c.ctx, gpu_runs, ref, weak)
                want = oracle.scalability(orc_runs, ref, weak)
                for r, (g, w) in enumerate(zip(got, want)):
                    assert g["trace_id"] == traces[r].trace_id and g["region"] == region
                    assert g["n_ranks"] == traces[r].n_ranks
                    for f in FIELDS:
                        assert bits(g[f]) == bits(w[f]), (region, ref, weak, r, f, g[f], w[f])
    st, _ = P.talp_gpu_scalability(c.ctx, gpu_runs, 7, False, check=False)
    assert st == -1
    mixed = [c.metrics(traces[0].trace_id, 0), c.metrics(traces[1].trace_id, 1)]
    st, _ = P.talp_gpu_scalability(c.ctx, mixed, 0, False, check=False)
    assert st == -1
    c.close()
