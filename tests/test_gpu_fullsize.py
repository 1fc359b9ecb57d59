"""Parity at full size in the launch configuration the benchmark times:
- the plain large trace (64 ranks x 4 GPUs x 4 streams, 2M device events per
  GPU, 1M host intervals per rank, 4 nested regions; 576M records; each
  device's 4 kernel streams are independent lanes, so kernels of different
  streams overlap and are merged by the flattening of Sec. 4.2);
- the scale trace (1024 ranks x 4 GPUs x 8 streams, bimodal kernels, 20% of
  ranks with 1.5x events; 1.10e9 records, 18.7 GB), generated in HBM by the
  generator's device twin;
each ingested from device memory with the start-order flag and the default
sweep shape.  The oracle reduces every unit of both traces (every rank's
host sums, every device's three unions, in every region, on the host cores:
rank by rank on threads) and the metrics of every region are compared with
the oracle's metrics formed from the oracle's own sums: every int64 field
exactly and every FP64 ratio bit for bit."""
import numpy as np
import pytest

import oracle
import tracegen as tg
from gpu_common import assert_metrics_equal

pytestmark = pytest.mark.gpu


def _compare_all(t_hdr, res, sums, hs_orc, du_orc, tag):
    """GPU unit sums and metrics vs the oracle's, every region."""
    for r in range(t_hdr.n_regions):
        np.testing.assert_array_equal(sums[r][0], hs_orc[r], err_msg=f"{tag}: host sums region {r}")
        np.testing.assert_array_equal(sums[r][1], du_orc[r], err_msg=f"{tag}: device unions region {r}")
        want = oracle.metrics_from_sums(t_hdr.n_ranks, t_hdr.devices_per_rank, hs_orc[r], du_orc[r],
                                        t_hdr.region_window[r])
        assert_metrics_equal(res[r], want, (tag, r))


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


def test_full_size_plain_every_unit_and_metric(full):
    t, res, sums = full
    assert t.n_records == 576_000_064
    first = np.concatenate([[0], np.cumsum(t.devices_per_rank.astype(np.int64))])

    def fetch(r0, r1):
        a, b = int(t.dev_off[first[r0]]), int(t.dev_off[first[r1]])
        return t.dev_se[a:b], t.dev_tag[a:b], t.dev_off[first[r0]:first[r1] + 1] - t.dev_off[first[r0]]

    du = oracle.device_unions_by_rank(fetch, t.n_ranks, t.devices_per_rank, t.region_window, block_ranks=16)
    hs = [oracle.host_sums(t, r) for r in range(t.n_regions)]
    _compare_all(t, res, sums, hs, du, "plain large")


def test_plain_large_kernels_overlap_across_streams(full):
    """The workload exercises the first flattening step of Sec. 4.2 (kernels
    of different streams overlapping): the union of kernels is well below
    their summed length on every device."""
    t, _, sums = full
    g0, g1 = int(t.dev_off[0]), int(t.dev_off[1])
    se, tag = t.dev_se[g0:g1], t.dev_tag[g0:g1]
    k = (tag >> 5) == 0
    assert len(np.unique(tag[k] & 31)) == 4
    summed = int((se[k, 1] - se[k, 0]).sum())
    assert sums[0][1][0, 0] < 0.9 * summed


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

    # the oracle over every device: the generated records (the generator's
    # output, the same input the GPU reduced) are copied out block by block
    def fetch(r0, r1):
        g0, g1 = int(first[r0]), int(first[r1])
        a, b = int(dt.dev_off[g0]), int(dt.dev_off[g1])
        return (dt.dev_se[a:b].cpu().numpy(), dt.dev_tag[a:b].cpu().numpy(),
                np.asarray(dt.dev_off[g0:g1 + 1], np.uint64) - np.uint64(a))

    du = oracle.device_unions_by_rank(fetch, spec.n_ranks, spec.devices_per_rank, dt.region_window,
                                      block_ranks=64)
    del arr, dt
    torch.cuda.empty_cache()
    return spec, T, res, sums, sampled, du


def _scale_host(spec, T):
    from tracegen import igen
    host = igen.host_trace(spec, T, ranks=[])          # windows of the whole trace
    win = igen.nested_regions(T, spec.n_regions)
    parts = [igen.host_lane(spec, i) for i in range(spec.n_ranks)]
    se = np.concatenate([np.concatenate([p[0], np.array([[p[2], max(int(T[i]), p[2])]], np.int64)])
                         for i, p in enumerate(parts)])
    st = np.concatenate([np.concatenate([p[1], np.array([1], np.uint8)]) for p in parts])
    off = np.zeros(spec.n_ranks + 1, np.uint64)
    off[1:] = np.cumsum(spec.host_events + 1)
    host.n_ranks, host.host_se, host.host_state, host.host_off, host.region_window = spec.n_ranks, se, st, off, win
    host.devices_per_rank = spec.devices_per_rank
    return host


def test_scale_full_size_every_unit_and_metric(scale_full):
    spec, T, res, sums, _, du = scale_full
    assert spec.n_records == 1_102_733_024       # 1.0e9 device records + 1024 x (100k + 1) host
    host = _scale_host(spec, T)
    hs = [oracle.host_sums(host, r) for r in range(spec.n_regions)]
    _compare_all(host, res, sums, hs, du, "scale")


def test_scale_generated_records_equal_the_host_twin(scale_full):
    """The device twin's records of sampled ranks equal the host twin's, and
    the oracle on the host twin's records gives the same unions."""
    from tracegen import igen
    spec, T, _, _, sampled, du = scale_full
    first = np.concatenate([[0], np.cumsum(spec.devices_per_rank.astype(np.int64))])
    for i in SCALE_SAMPLED_RANKS:
        t = igen.host_trace(spec, T, ranks=[i])
        np.testing.assert_array_equal(sampled[i][0], t.dev_se, err_msg=f"generated records of rank {i}")
        np.testing.assert_array_equal(sampled[i][1], t.dev_tag)
        g0, g1 = int(first[i]), int(first[i + 1])
        for r in range(spec.n_regions):
            np.testing.assert_array_equal(du[r][g0:g1], oracle.device_unions(t, r), err_msg=f"rank {i} region {r}")
