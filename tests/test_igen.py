"""The counter-based generator's host twin: lane structure, laws, and the
shortcut used for rank ends (no GPU; the device twin is compared with this
one in test_gpu_igen.py)."""
import numpy as np
import pytest

from tracegen import igen


def test_vector_keys_match_scalar_keys():
    ks = igen.unit_keys(11, 7, igen.DOM_DEV, np.arange(100))
    assert [int(k) for k in ks] == [igen.unit_key(11, 7, igen.DOM_DEV, i) for i in range(100)]


def _spec(E, law=igen.LAW_LOGNORMAL, ks=1, H=50):
    return igen.TraceSpec(trace_id=3, seed=5, devices_per_rank=np.array([len(E)], np.uint32),
                          dev_events=np.asarray(E, np.int64), host_events=np.array([H], np.int64),
                          work_milli=np.array([850], np.int64), law=law, n_kstreams=ks, copy_stream0=ks,
                          n_cstreams=2, n_regions=3)


@pytest.mark.parametrize("E", [1, 2, 3, 7, 10, 1000, 33333])
def test_device_lane_structure(E):
    sp = _spec([E], ks=3)
    se, tag = igen.device_lane(sp, 0)
    assert se.shape == (E, 2) and tag.shape == (E,)
    assert np.all(np.diff(se[:, 0]) >= 0)                    # start order by construction
    assert np.all(se[:, 1] > se[:, 0])
    kinds = tag >> 5
    S = (7 * E + 5) // 10
    assert int((kinds == 0).sum()) == S and int((kinds != 0).sum()) == E - S
    assert set(np.unique(kinds)) <= {0, 1, 2}
    assert set(np.unique(tag[kinds == 0] & 31)) <= {0, 1, 2}
    assert set(np.unique(tag[kinds != 0] & 31)) <= {3, 4}
    # kernels never overlap each other (one timeline)
    k = se[kinds == 0]
    assert np.all(k[1:, 0] >= k[:-1, 1])
    assert igen.device_lane_end(sp, 0) == int(se[:, 1].max())


def test_lane_end_shortcut_on_many_lanes():
    sp = _spec(list(range(1, 60)) + [5000, 20000], law=igen.LAW_BIMODAL, ks=6)
    for g in range(sp.m_devices):
        se, _ = igen.device_lane(sp, g)
        assert igen.device_lane_end(sp, g) == int(se[:, 1].max()), g


def test_laws():
    sp = _spec([400000], H=200000)
    se, tag = igen.device_lane(sp, 0)
    k = se[(tag >> 5) == 0]
    d = k[:, 1] - k[:, 0]
    # lognormal(ln 20 us, 1) times the work factor 0.85 (table-quantised)
    assert abs(d.mean() / (igen.MEAN_KERNEL_NS[igen.LAW_LOGNORMAL] * 0.85) - 1) < 0.03
    assert abs(np.median(d) / (20_000 * 0.85) - 1) < 0.03
    # kernel occupancy of the lane ~ 0.7
    span = se[:, 1].max() - se[:, 0].min()
    assert abs(d.sum() / span - 0.7) < 0.02
    hs, st, end = igen.host_lane(sp, 0)
    assert np.all(hs[1:, 0] == hs[:-1, 1]) and hs[0, 0] == 0 and end == hs[-1, 1]
    for s, mean in enumerate((50_000, 5_000, 10_000)):
        dur = (hs[:, 1] - hs[:, 0])[st == s]
        assert abs(dur.mean() / mean - 1) < 0.03
        assert abs((st == s).mean() - 1 / 3) < 0.01


def test_host_trace_tiles_and_pads_to_rank_end():
    sp = igen.scale_spec(scale=0.001, n_ranks=6)
    T = igen.rank_ends(sp, threads=2)
    t = igen.host_trace(sp, T)
    for i in range(t.n_ranks):
        a, b = int(t.host_off[i]), int(t.host_off[i + 1])
        h = t.host_se[a:b]
        assert h[0, 0] == 0 and np.all(h[1:, 0] == h[:-1, 1]) and h[-1, 1] == T[i]
        assert t.host_state[b - 1] == 1
    np.testing.assert_array_equal(t.region_window[0, :, 1], T)
    sub = igen.host_trace(sp, T, ranks=[2, 3])
    np.testing.assert_array_equal(sub.region_window, t.region_window[:, 2:4])
    a0, a1 = int(t.dev_off[8]), int(t.dev_off[16])
    np.testing.assert_array_equal(sub.dev_se, t.dev_se[a0:a1])


def test_waves_group_whole_traces():
    specs = igen.batched_specs(n_traces=40, ev_lo=10, ev_hi=1000, max_ranks=16)
    ws = igen.waves(specs, 50_000)
    assert [sp.trace_id for w in ws for sp in w] == list(range(40))
    for w in ws:
        assert len(w) == 1 or sum(sp.n_records for sp in w) <= 50_000


def test_plain_large_has_concurrent_kernel_streams():
    """The plain large trace's 4 kernel streams are independent lanes: on a
    device, kernels of different streams overlap (up to 4 at once), so the
    headline workload merges concurrent kernels as Sec. 4.2's first
    flattening step requires.  Counted by a +1/-1 sweep over the events of
    two devices of a 1% sample (same laws, fewer events)."""
    import tracegen as tg
    t = tg.plain_large(scale=0.01, n_ranks=2, gpus_per_rank=1)
    for g in range(t.m_devices):
        a, b = int(t.dev_off[g]), int(t.dev_off[g + 1])
        se, tag = t.dev_se[a:b], t.dev_tag[a:b]
        k = (tag >> 5) == 0
        assert sorted(np.unique(tag[k] & 31)) == [0, 1, 2, 3]
        pts = np.concatenate([se[k, 0], se[k, 1]])
        step = np.concatenate([np.ones(int(k.sum()), np.int64), -np.ones(int(k.sum()), np.int64)])
        order = np.lexsort((step, pts))                     # ends before starts at equal times
        level = np.cumsum(step[order])
        assert level.max() == 4
        # time with two or more kernels running: a sizeable share of the kernel time
        dt = np.diff(pts[order])
        multi = int(dt[level[:-1] >= 2].sum())
        assert multi > 0.1 * int((se[k, 1] - se[k, 0]).sum())
