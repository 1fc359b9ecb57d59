"""Parity at full size in the launch configuration the benchmark times:
- the plain large trace (64 ranks x 4 GPUs x 4 streams, 2M device events per
  GPU, 1M host intervals per rank, 4 nested regions; 576M records);
- the scale trace (1024 ranks x 4 GPUs x 8 streams, bimodal kernels, 20% of
  ranks with 1.5x events; 1.10e9 records, 18.7 GB), generated in HBM by the
  generator's device twin;
each ingested from device memory with the start-order flag and the default
sweep shape.  The oracle checks every rank's host sums and the host half of
every region's metrics exactly, the unions of the devices of sampled ranks
exactly, and the device half through properties that hold at any size."""
import numpy as np
import pytest

import oracle
import tracegen as tg
from paper_2603_26576_b300 import shard

pytestmark = pytest.mark.gpu

SAMPLED_RANKS = (0, 37, 63)


@pytest.fixture(scope="module")
def full():
    import torch
    import paper_2603_26576_b300 as P
    t = tg.plain_large()
    dev = torch.device("cuda", 0)
    arr = dict(host_se=torch.from_numpy(t.host_se).to(dev), host_state=torch.from_numpy(t.host_state).to(dev),
               dev_se=torch.from_numpy(t.dev_se).to(dev), dev_tag=torch.from_numpy(t.dev_tag).to(dev))
    ctx = P.Context(0)
    ctx.ingest([t], flags=P.TALP_GPU_SORTED_BY_START, arrays=[arr])
    res = ctx.metrics(t.trace_id)
    sums = [ctx.unit_sums(t.trace_id, r) for r in range(t.n_regions)]
    ctx.close()
    del arr
    torch.cuda.empty_cache()
    return t, res, sums


def _check_host(t, res, sums, hs_of):
    for r in range(t.n_regions):
        hs = hs_of(r)
        np.testing.assert_array_equal(sums[r][0], hs, err_msg=f"host sums region {r}")
        tot = hs.sum(axis=1)
        assert res[r]["elapsed_ns"] == int(tot.max())                      # Eq. 1
        assert res[r]["sum_useful"] == int(hs[:, 0].sum())
        assert res[r]["sum_offload"] == int(hs[:, 1].sum())
        assert res[r]["sum_mpi"] == int(hs[:, 2].sum())
        assert res[r]["max_useful_offload"] == int((hs[:, 0] + hs[:, 1]).max())


def test_full_size_host_sums_and_host_metrics(full):
    t, res, sums = full
    assert t.n_records == 576_000_064
    _check_host(t, res, sums, lambda r: oracle.host_sums(t, r))


def test_full_size_sampled_device_unions(full):
    t, _, sums = full
    first_dev = np.concatenate([[0], np.cumsum(t.devices_per_rank.astype(np.int64))])
    for i in SAMPLED_RANKS:
        s = shard.shard_of(t, [i])
        g0, g1 = int(first_dev[i]), int(first_dev[i + 1])
        for r in range(t.n_regions):
            np.testing.assert_array_equal(sums[r][1][g0:g1], oracle.device_unions(s, r),
                                          err_msg=f"rank {i} region {r}")


def test_full_size_device_metrics_properties(full):
    t, res, sums = full
    _check_device_properties(t, res, sums)


def _check_device_properties(t, res, sums):
    for r in range(t.n_regions):
        m = res[r]
        d = sums[r][1]
        K, UM, B = d[:, 0], d[:, 1], d[:, 2]
        win = t.region_window[r][np.repeat(np.arange(t.n_ranks), t.devices_per_rank)]
        assert np.all(K <= B) and np.all(UM <= B) and np.all(B <= K + UM)   # union <= sum
        assert np.all(B <= win[:, 1] - win[:, 0])
        assert m["sum_kernel"] == int(K.sum()) and m["max_kernel"] == int(K.max())
        assert m["max_busy"] == int(B.max()) and m["sum_mem"] == int((B - K).sum())
        assert m["sum_hidden_mem"] == int((K + UM - B).sum())
        assert m["sum_idle"] == int(((win[:, 1] - win[:, 0]) - B).sum())
        for f in ("host_pe", "host_mpi_pe", "host_mpi_lb", "host_mpi_ce", "host_oe", "dev_pe", "dev_lb", "dev_ce",
                  "dev_oe"):
            assert 0.0 <= m[f] <= 1.0, (r, f, m[f])
        # each parent is the product of its children (Eqs. 6-12), to rounding
        assert abs(m["dev_pe"] - m["dev_lb"] * m["dev_ce"] * m["dev_oe"]) <= 4 * np.spacing(m["dev_pe"])
        assert abs(m["host_mpi_pe"] - m["host_mpi_lb"] * m["host_mpi_ce"]) <= 4 * np.spacing(m["host_mpi_pe"])
        assert abs(m["host_pe"] - m["host_mpi_pe"] * m["host_oe"]) <= 4 * np.spacing(m["host_pe"])
        # the ratios are the FP64 expressions of these exact aggregates
        E, n, mm = m["elapsed_ns"], t.n_ranks, t.m_devices
        assert m["dev_pe"] == float(m["sum_kernel"]) / (float(E) * float(mm))
        assert m["dev_lb"] == float(m["sum_kernel"]) / (float(mm) * float(m["max_kernel"]))
        assert m["dev_ce"] == float(m["max_kernel"]) / float(m["max_busy"])
        assert m["dev_oe"] == float(m["max_busy"]) / float(E)
        assert m["host_pe"] == float(m["sum_useful"]) / (float(E) * float(n))


# ---------------------------------------------------------------- scale trace

SCALE_SAMPLED_RANKS = (0, 511, 1023)


@pytest.fixture(scope="module")
def scale_full():
    import torch
    import paper_2603_26576_b300 as P
    from tracegen import igen
    spec = igen.scale_spec()
    T = igen.rank_ends(spec)
    (dt,) = igen.generate_device([spec])
    arr = dict(host_se=dt.host_se, host_state=dt.host_state, dev_se=dt.dev_se, dev_tag=dt.dev_tag)
    ctx = P.Context(0)
    ctx.ingest([dt], flags=P.TALP_GPU_SORTED_BY_START, arrays=[arr])
    res = ctx.metrics(dt.trace_id)
    sums = [ctx.unit_sums(dt.trace_id, r) for r in range(dt.n_regions)]
    ctx.close()
    first = np.concatenate([[0], np.cumsum(spec.devices_per_rank.astype(np.int64))])
    sampled = {}
    for i in SCALE_SAMPLED_RANKS:
        a, b = int(dt.dev_off[first[i]]), int(dt.dev_off[first[i + 1]])
        sampled[i] = (dt.dev_se[a:b].cpu().numpy(), dt.dev_tag[a:b].cpu().numpy())
    del arr, dt
    torch.cuda.empty_cache()
    return spec, T, res, sums, sampled


def test_scale_full_size_host(scale_full):
    from tracegen import igen
    spec, T, res, sums, _ = scale_full
    assert spec.n_records == 1_102_733_024       # 1.0e9 device records + 1024 x (100k + 1) host
    host = igen.host_trace(spec, T, ranks=[])          # windows of the whole trace
    win = igen.nested_regions(T, spec.n_regions)
    parts = [igen.host_lane(spec, i) for i in range(spec.n_ranks)]
    se = np.concatenate([np.concatenate([p[0], np.array([[p[2], max(int(T[i]), p[2])]], np.int64)])
                         for i, p in enumerate(parts)])
    st = np.concatenate([np.concatenate([p[1], np.array([1], np.uint8)]) for p in parts])
    off = np.zeros(spec.n_ranks + 1, np.uint64)
    off[1:] = np.cumsum(spec.host_events + 1)
    host.n_ranks, host.host_se, host.host_state, host.host_off, host.region_window = spec.n_ranks, se, st, off, win
    _check_host(host, res, sums, lambda r: oracle.host_sums(host, r))


def test_scale_full_size_sampled_devices(scale_full):
    from tracegen import igen
    spec, T, _, sums, sampled = scale_full
    first = np.concatenate([[0], np.cumsum(spec.devices_per_rank.astype(np.int64))])
    for i in SCALE_SAMPLED_RANKS:
        t = igen.host_trace(spec, T, ranks=[i])
        np.testing.assert_array_equal(sampled[i][0], t.dev_se, err_msg=f"generated records of rank {i}")
        np.testing.assert_array_equal(sampled[i][1], t.dev_tag)
        g0, g1 = int(first[i]), int(first[i + 1])
        for r in range(spec.n_regions):
            np.testing.assert_array_equal(sums[r][1][g0:g1], oracle.device_unions(t, r),
                                          err_msg=f"rank {i} region {r}")


def test_scale_full_size_device_properties(scale_full):
    from tracegen import igen
    spec, T, res, sums, _ = scale_full
    t = igen.host_trace(spec, T, ranks=[])
    t.n_ranks, t.devices_per_rank = spec.n_ranks, spec.devices_per_rank
    t.region_window = igen.nested_regions(T, spec.n_regions)
    t.dev_off = np.zeros(spec.m_devices + 1, np.uint64)
    _check_device_properties(t, res, sums)
