"""The generator's device twin reproduces the host twin bit for bit, and the
reduction of device-generated traces equals the oracle on the host twin's
copy of them."""
import numpy as np
import pytest

import oracle
from gpu_common import assert_metrics_equal, make_ctx
from tracegen import igen

pytestmark = pytest.mark.gpu


def _specs():
    sp = igen.batched_specs(n_traces=30, ev_lo=1, ev_hi=3000, max_ranks=12, max_gpus=4)
    sp.append(igen.scale_spec(scale=0.002, n_ranks=10, trace_id=777))
    return sp


def test_device_twin_equals_host_twin():
    specs = _specs()
    dts = igen.generate_device(specs)
    for sp, dt in zip(specs, dts):
        T = igen.rank_ends(sp, threads=4)
        np.testing.assert_array_equal(dt.T, T, err_msg=f"rank ends of trace {sp.trace_id}")
        t = igen.host_trace(sp, T)
        np.testing.assert_array_equal(dt.region_window, t.region_window)
        np.testing.assert_array_equal(dt.host_off, t.host_off)
        np.testing.assert_array_equal(dt.dev_off, t.dev_off)
        np.testing.assert_array_equal(dt.host_se.cpu().numpy(), t.host_se, err_msg=str(sp.trace_id))
        np.testing.assert_array_equal(dt.host_state.cpu().numpy(), t.host_state)
        np.testing.assert_array_equal(dt.dev_se.cpu().numpy(), t.dev_se, err_msg=str(sp.trace_id))
        np.testing.assert_array_equal(dt.dev_tag.cpu().numpy(), t.dev_tag)


def test_plan_over_generated_traces_matches_oracle():
    import paper_2603_26576_b300 as P
    specs = _specs()
    dts = igen.generate_device(specs)
    c = make_ctx()
    arrays = [dict(host_se=d.host_se, host_state=d.host_state, dev_se=d.dev_se, dev_tag=d.dev_tag) for d in dts]
    plan = c.plan(dts, arrays, flags=P.TALP_GPU_SORTED_BY_START)
    plan.launch()
    res = plan.metrics()
    q = 0
    for sp, dt in zip(specs, dts):
        t = igen.host_trace(sp, dt.T)
        for r in range(sp.n_regions):
            assert res[q]["trace_id"] == sp.trace_id and res[q]["region"] == r
            assert_metrics_equal(res[q], oracle.region_metrics(t, r), ("igen plan", sp.trace_id, r))
            q += 1
    plan.close()
    c.close()
