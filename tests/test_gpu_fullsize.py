"""Parity at full size in the launch configuration the benchmark times: the
plain large trace (64 ranks x 4 GPUs x 4 streams, 2M device events per GPU,
1M host intervals per rank, 4 nested regions; 576M records) ingested from
device memory with the start-order flag and the default sweep shape.
The oracle checks every rank's host sums and the host half of every
region's metrics exactly, the unions of the devices of sampled ranks
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


def test_full_size_host_sums_and_host_metrics(full):
    t, res, sums = full
    assert t.n_records == 576_000_064
    for r in range(t.n_regions):
        hs = oracle.host_sums(t, r)
        np.testing.assert_array_equal(sums[r][0], hs, err_msg=f"host sums region {r}")
        tot = hs.sum(axis=1)
        assert res[r]["elapsed_ns"] == int(tot.max())                      # Eq. 1
        assert res[r]["sum_useful"] == int(hs[:, 0].sum())
        assert res[r]["sum_offload"] == int(hs[:, 1].sum())
        assert res[r]["sum_mpi"] == int(hs[:, 2].sum())
        assert res[r]["max_useful_offload"] == int((hs[:, 0] + hs[:, 1]).max())


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
