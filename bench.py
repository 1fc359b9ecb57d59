#!/usr/bin/env python3
"""Benchmark of the efficiency-metric reducer on synthetic traces.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]
                  [--workload plain|small|scale|batched|batched-full|serving|concurrency|raw|threads]
                  [--scale S]

One step = one pass of the whole hot path over one trace resident in HBM:
record validation, the device flattening (kernel / transfer / busy unions per
device and region), the host-state sums, and the final reduction into the
nine efficiency ratios of every region (launched through the C ABI).

Default workload ("plain"): one trace of 64 ranks x 4 GPUs x 4 streams,
2M device events per GPU and 1M host intervals per rank, 4 nested regions
(576M records, 9.8 GB), generated seeded on the host.  Its inputs are far
larger than the 126 MB L2, so no flush is needed between steps.

value   : records (events) per second with the inputs already in HBM;
e2e     : the same metric through the C ABI from pinned HOST buffers, the
          host->device copy of every step's records and the device->host
          copy of its metrics inside the timed region;
roofline: the sweep kernel (the dominant kernel) against the measured HBM
          copy bandwidth: 17 algorithmic bytes per record / its CUDA-event
          duration (with --unsorted: the sort stage, 17 bytes per device
          record / its CUDA-event duration);
cpu_baseline: the CPU oracle on a bounded one-rank sample of the workload.

The default command's line also carries sub-objects measured in the same
run: `serving` and `serving_plain` (the served form and the plain form at
the serving load: p50/p99 query latency, the served form's both from Python
client threads and from native client threads that call the C ABI, and
inside the library), `batched` (the small-trace batched
form against one trace per launch), `sort_stage` (the same trace with each
device's records grouped by stream, sorted by the library), `concurrency`
(the concurrency profile of its devices) and `raw` (the trace at 25% as raw
activity-record buffers), each with its own exactness check and clocks.

--impl reference times the CPU oracle itself (the slow, plain statement of
the method) on a bounded sample per step; it is the reference arm.

With N > 1 (torchrun, one rank per GPU) every rank reduces its own trace of
the same shape (weak scaling, no collective on the data path); the timing is
the max over ranks.
"""
import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import tracegen as tg  # noqa: E402

METRIC = "events/s and HBM GB/s for host+device efficiency metrics; p99 runtime-query ms"
UNIT = "events/s"
BYTES_PER_RECORD = 17


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="plain",
                    choices=["plain", "small", "scale", "batched", "batched-full", "serving", "concurrency", "raw",
                             "threads"])
    ap.add_argument("--wave-records", type=float, default=3e9, help="batched-full: records per wave")
    ap.add_argument("--traces", type=int, default=4096, help="batched: number of traces")
    ap.add_argument("--check-wave", type=int, default=None,
                    help="batched-full: the wave checked whole against the oracle (default: the smallest of >= 16 traces)")
    ap.add_argument("--ev-hi", type=int, default=None,
                    help="batched: largest events per GPU (default 5000; batched-full 1e6)")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--jobs", type=int, default=256, help="serving: monitored jobs")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: batch arrivals per second (all jobs)")
    ap.add_argument("--query-ms", type=float, default=10.0, help="serving: query period per job")
    ap.add_argument("--step-s", type=float, default=1.0, help="serving: seconds of served load per step")
    ap.add_argument("--sat-s", type=float, default=3.0, help="serving: seconds of the saturation phase")
    ap.add_argument("--plain-s", type=float, default=3.0, help="serving: seconds of the plain-form phase")
    ap.add_argument("--native-s", type=float, default=5.0,
                    help="serving: seconds of the same load from native client threads (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grouped-hint", action="store_true",
                    help="with --unsorted: pass TALP_GPU_GROUPED_BY_STREAM (the caller states its device records come "
                         "grouped by stream, each group in start order)")
    ap.add_argument("--not-sorted-hint", action="store_true",
                    help="with --unsorted: pass TALP_GPU_NOT_SORTED (the caller knows its records are out of order)")
    ap.add_argument("--unsorted", action="store_true",
                    help="plain/small: device records grouped by stream (each stream in start order, as per-stream "
                         "activity buffers deliver them); the library sorts them")
    ap.add_argument("--runs", type=int, default=0,
                    help="with --unsorted: deal each device's records into this many sorted runs laid end to end "
                         "instead of grouping them by stream")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="plain: skip the serving, plain-serving and batched sub-objects of the default line")
    ap.add_argument("--hold-calls", type=int, default=1,
                    help="raw: stream each step's records as this many delivery buffers with hold-back")
    return ap.parse_args()


def workload(name, scale, rank):
    if name == "scale":
        from tracegen import igen
        spec = igen.scale_spec(seed=0x7A1F + 3 + 1000 * rank, scale=scale, trace_id=3 + rank)
        desc = "scale trace: 1024 ranks x 4 GPUs x 8 streams, bimodal kernels, 20% of ranks with 1.5x events, " \
               "222k device events/GPU, 100k host intervals/rank, 4 nested regions (generated in HBM)"
        return spec, desc
    if name == "plain":
        t = tg.plain_large(seed=0x7A1F + 1 + 1000 * rank, scale=scale, trace_id=1 + rank)
        desc = "plain large single trace: 64 ranks x 4 GPUs x 4 streams, 2M device events/GPU, " \
               "1M host intervals/rank, 4 nested regions"
    else:
        t = tg.single_trace_small(seed=0x7A1F + 1000 * rank, scale=scale, trace_id=rank)
        desc = "single trace: 4 ranks x 1 GPU x 1 stream, 10k host + 10k device intervals/rank, 1 region"
    return t, desc


def oracle_sample(name, scale):
    """A bounded sample of the workload for the CPU oracle: one rank of it."""
    if name == "scale":
        from tracegen import igen
        spec = igen.scale_spec(scale=scale)
        T = igen.rank_ends(spec)
        heavy = int(np.argmax(spec.dev_events[::4]))
        return igen.host_trace(spec, T, ranks=[heavy])
    if name == "plain":
        return tg.plain_large(seed=0x7A1F + 1, scale=scale, trace_id=1, n_ranks=1)
    return tg.single_trace_small(scale=scale)


def host_cpu():
    """The host the CPU oracle runs on: logical cores and CPU model."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"host_nproc": os.cpu_count(), "host_cpu": model}


def _oracle_worker(args):
    """One process of the all-cores oracle run: the same bounded sample,
    timed three times (the median), so that the processes overlap."""
    name, scale = args
    import oracle
    s = oracle_sample(name, scale)
    dts = sorted(time_oracle(s) for _ in range(3))
    return s.n_records, dts[1]


def oracle_all_cores(name, scale):
    """The untuned oracle on every host core at once: one process per core
    (started by spawn: this process holds a GPU context), each on the
    sample; the throughput is the sum over processes."""
    import multiprocessing as mp
    p = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(p) as pool:
        res = pool.map(_oracle_worker, [(name, scale)] * p)
    return sum(n / dt for n, dt in res), p, res[0][0]


def time_oracle(t):
    import oracle
    t0 = time.perf_counter()
    for r in range(t.n_regions):
        oracle.host_sums(t, r)
        oracle.device_unions(t, r)
    return time.perf_counter() - t0


class Clocks:
    """nvidia-smi sampler for the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    # The samples go to a temporary file, read at stop(): a Python thread
    # reading a pipe from nvidia-smi slowed a host-synchronising step by ~15%.
    def _read_file(self):
        self.out.seek(0)
        return [ln.strip() for ln in self.out.read().splitlines() if ln.strip()]

    def start(self):
        import tempfile
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        # the file is read only after nvidia-smi has exited (the two share
        # its offset); the warm-up that follows (warm_until) covers its start

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait(timeout=5)
        self.lines = self._read_file()
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def warm_until(fn, n_min, seconds=1.0):
    """Untimed warm-up: at least n_min steps, and steps until `seconds` of
    wall time have passed, so that the timed steps follow continuous work.
    After an idle spell (or nvidia-smi's start) the first ~100 ms of
    host-synchronising round trips ran up to 3x slower on the B300 machines."""
    import torch
    t0 = time.perf_counter()
    k = 0
    while k < n_min or time.perf_counter() - t0 < seconds:
        fn()
        k += 1
        if k % 4 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    return k


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def sweep_traffic_per_record():
    """dram bytes per record of the sweep kernel from the committed ncu
    summary, valid only while the kernel source is unchanged."""
    src = os.path.join(ROOT, "paper_2603_26576_b300", "csrc", "sweep.cu")
    prof = os.path.join(ROOT, "profiles", "sweep_plain_large.txt")
    if not os.path.exists(prof):
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    kv = {}
    for ln in open(prof):
        if ":" in ln:
            k, v = ln.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("sweep_source_sha256_16") != h:
        return None
    try:
        return float(kv["dram_bytes_per_record"])
    except (KeyError, ValueError):
        return None


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(a):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    t = oracle_sample(a.workload, a.scale if a.workload == "small" else min(a.scale, 1.0))
    n = t.n_records
    for _ in range(a.warmup):
        time_oracle(t)
    dts = [time_oracle(t) for _ in range(a.steps)]
    total = sum(dts)
    value = n * a.steps / total
    _, desc = (None, "")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1000 * total / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic (seeded generator)", "impl": "reference",
        "config": {"workload": workload_name(a), "sample": f"one rank of the workload: {n} records per step",
                   "l2": "inputs in host memory (CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"one rank ({t.m_devices} devices, {n} records) x {t.n_regions} regions",
                         **host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_name(a):
    if a.workload == "plain":
        base = "plain large single trace: 64 ranks x 4 GPUs x 4 streams, 2M device events/GPU, 1M host intervals/rank, 4 nested regions"
    elif a.workload == "scale":
        base = ("scale trace: 1024 ranks x 4 GPUs x 8 streams, bimodal kernels (1 us / 500 us, 80/20), 20% of ranks "
                "with 1.5x events, 222k device events/GPU, 100k host intervals/rank, 4 nested regions")
    else:
        base = "single trace: 4 ranks x 1 GPU x 1 stream, 10k host + 10k device intervals/rank, 1 region"
    if a.unsorted:
        base += (f", each device's records in {a.runs} sorted runs (sorted by the library)" if getattr(a, "runs", 0)
                 else ", device records grouped by stream (sorted by the library)")
    return base if a.scale == 1.0 else f"{base} (scale {a.scale})"


def run_batched(a):
    line = measure_batched(a)
    print(json.dumps(line), flush=True)
    return 0 if line["config"]["bit_exact_batched_vs_plain"] and line["config"]["bit_exact_sampled_vs_oracle"] else 1


def measure_batched(a):
    """Batched form: thousands of uneven traces reduced by one CUDA-graph
    launch of an autotuned plan, against one ingest + finalize per trace.
    Every trace's metrics of the two forms are compared bit for bit, and 16
    traces spread over the workload against the oracle."""
    import torch
    import oracle
    import paper_2603_26576_b300 as P
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    t0 = time.time()
    ev_hi = a.ev_hi or 5000
    ts = tg.batched_workload(n_traces=a.traces, ev_lo=5, ev_hi=ev_hi)
    gen_s = time.time() - t0
    N = sum(t.n_records for t in ts)
    # one device buffer per record array; each trace a 16-byte aligned view
    def pack(field, dt, width):
        sizes = [getattr(t, field).shape[0] for t in ts]
        offs = np.zeros(len(ts) + 1, np.int64)
        offs[1:] = np.cumsum([(s + 15) // 16 * 16 for s in sizes])
        buf = torch.empty((int(offs[-1]),) + ((width,) if width > 1 else ()), dtype=dt, device=dev)
        for k, t in enumerate(ts):
            arr = torch.from_numpy(np.ascontiguousarray(getattr(t, field)))
            buf[int(offs[k]):int(offs[k]) + sizes[k]].copy_(arr)
        return [buf[int(offs[k]):int(offs[k]) + sizes[k]] for k in range(len(ts))], buf
    hse, b1 = pack("host_se", torch.int64, 2)
    hst, b2 = pack("host_state", torch.uint8, 1)
    dse, b3 = pack("dev_se", torch.int64, 2)
    dtg, b4 = pack("dev_tag", torch.uint8, 1)
    arrays = [dict(host_se=hse[k], host_state=hst[k], dev_se=dse[k], dev_tag=dtg[k]) for k in range(len(ts))]
    torch.cuda.synchronize()
    ctx = P.Context(0)
    stream = torch.cuda.Stream(device=dev)
    t1 = time.time()
    plan = ctx.plan(ts, arrays, flags=P.TALP_GPU_SORTED_BY_START, plan_flags=P.TALP_GPU_PLAN_AUTOTUNE)
    plan_s = time.time() - t1
    info = plan.info()
    clocks = Clocks(0)
    clocks.start()
    warm_until(lambda: plan.launch(stream), max(a.warmup, 3))
    batched = plan.metrics(stream)
    P.talp_gpu_profile_read(ctx.ctx)
    l0 = P.talp_gpu_profile_read(ctx.ctx)["kernel_launches"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        plan.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    launches = P.talp_gpu_profile_read(ctx.ctx)["kernel_launches"] - l0
    # plain form: one ingest + one finalize per trace, same traces, same GPU
    batches = []
    for t, arr in zip(ts, arrays):
        b, keep = P.batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, arr["host_se"],
                                      arr["host_state"], t.host_off, arr["dev_se"], arr["dev_tag"], t.dev_off,
                                      P.TALP_GPU_SORTED_BY_START)
        batches.append((b, keep, t))
    out_dev = torch.empty(8 * 200, dtype=torch.uint8, device=dev)

    def plain_pass():
        for b, _, t in batches:
            P.talp_gpu_ingest_events(ctx.ctx, [b], stream)
            P.talp_gpu_region_metrics_device(ctx.ctx, [t.trace_id], P.TALP_GPU_ALL_REGIONS, out_dev.data_ptr(),
                                             stream)
    plain_pass()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    plain_pass()
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - w0
    # bit-exact agreement of the two forms
    plain_res = []
    for _, _, t in batches:
        plain_res += [P.metrics_to_dict(x) for x in
                      P.talp_gpu_region_metrics(ctx.ctx, t.trace_id, P.TALP_GPU_ALL_REGIONS, stream,
                                                n_regions=t.n_regions)]
    agree = plain_res == batched
    # the oracle on 16 traces spread over the workload, every region
    firsts = np.concatenate([[0], np.cumsum([t.n_regions for t in ts])])
    sampled = sorted(set(int(k) for k in np.linspace(0, len(ts) - 1, 16)))
    exact = True
    cpu_rec, cpu_s = 0, 0.0
    for k in sampled:
        c0 = time.perf_counter()
        ref = oracle.trace_metrics(ts[k])
        cpu_s += time.perf_counter() - c0
        cpu_rec += ts[k].n_records
        for r in range(ts[k].n_regions):
            got = batched[int(firsts[k]) + r]
            for f in oracle.INT_FIELDS + oracle.RATIO_FIELDS:
                exact &= got[f] == ref[r][f]
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_RECORD * N / (ms / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": N / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic (seeded generator; the paper's traces are not available)",
        "config": {"workload": f"batched: {len(ts)} traces, ranks log-uniform 1-512, 1-8 GPUs per rank, "
                               f"5-{ev_hi} device events per GPU log-uniform, 8 nested regions each",
                   "form": "one CUDA-graph launch of an autotuned plan per step", "records_per_step": N,
                   "plan": info, "plan_build_s": plan_s, "generate_s": gen_s,
                   "plain_one_trace_per_launch_events_per_s": N / plain_s,
                   "batched_over_plain": (N / (ms / 1000.0)) / (N / plain_s),
                   "bit_exact_batched_vs_plain": agree,
                   "oracle_sampled_traces": sampled, "bit_exact_sampled_vs_oracle": bool(exact),
                   "l2": "inputs (%.1f GB) larger than L2; no flush" % (BYTES_PER_RECORD * N / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "whole graph (prep, sweep, fixup, finalize)", "kernel_ms": ms,
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "cpu_baseline": {"value": cpu_rec / cpu_s if cpu_s else None, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"the {len(sampled)} traces checked ({cpu_rec} records), {cpu_s:.2f} s"},
        "e2e": None, "gpu_launches": launches, "clocks": ck,
    }
    plan.close()
    ctx.close()
    del arrays, hse, hst, dse, dtg, b1, b2, b3, b4, batches
    torch.cuda.empty_cache()
    return line


def run_batched_full(a):
    """The batched workload at its full laws (4096 traces, 1e3-1e6 device
    events per GPU: 2.6e11 records, 4.3 TB), far beyond HBM: consecutive
    waves of whole traces are generated in HBM by the generator's device
    twin (untimed), each wave is reduced by one CUDA-graph launch of a plan
    (timed with CUDA events) and, for comparison, by one ingest + finalize
    per trace.  The smallest trace of every wave is checked against the
    oracle on the host twin's copy of it."""
    import torch
    import oracle
    import paper_2603_26576_b300 as P
    from tracegen import igen
    torch.cuda.set_device(0)
    ev_hi = a.ev_hi or 1_000_000
    specs = igen.batched_specs(n_traces=a.traces, ev_hi=ev_hi)
    wv = igen.waves(specs, int(a.wave_records))
    stream = torch.cuda.Stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tot_rec = tot_seg = 0
    plan_ms = plain_ms = gen_s = build_s = 0.0
    launches = 0
    exact = True
    checked = []
    cpu_rec, cpu_s = 0, 0.0
    # the wave checked whole against the oracle: the one with the fewest
    # records among the waves of at least 16 traces (or the fewest overall)
    wrec = [sum(sp.n_records for sp in w) for w in wv]
    big = [i for i, w in enumerate(wv) if len(w) >= 16] or list(range(len(wv)))
    check_wave = a.check_wave if a.check_wave is not None else min(big, key=lambda i: wrec[i])
    whole_rec, whole_traces, whole_s = 0, 0, 0.0
    ctx = P.Context(0)
    clocks = Clocks(0)
    clocks.start()
    out_dev = torch.empty(8 * 200, dtype=torch.uint8, device="cuda")
    for wi, w in enumerate(wv):
        g0 = time.perf_counter()
        dts = igen.generate_device(w, stream=stream)
        torch.cuda.synchronize()
        gen_s += time.perf_counter() - g0
        arrays = [dict(host_se=d.host_se, host_state=d.host_state, dev_se=d.dev_se, dev_tag=d.dev_tag) for d in dts]
        b0 = time.perf_counter()
        plan = ctx.plan(dts, arrays, flags=P.TALP_GPU_SORTED_BY_START)
        build_s += time.perf_counter() - b0
        info = plan.info()
        # warm-up (and first result): the wave was just generated and planned
        warm_until(lambda: plan.launch(stream), 2, 0.15)
        e0.record(stream)
        for _ in range(3):
            plan.launch(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        plan_ms += e0.elapsed_time(e1) / 3
        launches += 3 * info["kernels_per_launch"]
        res = plan.metrics(stream)
        # plain form on the same wave: one ingest + one finalize per trace
        batches = []
        for d, arr in zip(dts, arrays):
            b, keep = P.batch_from_arrays(d.trace_id + (1 << 40), d.devices_per_rank, d.region_window,
                                          arr["host_se"], arr["host_state"], d.host_off, arr["dev_se"],
                                          arr["dev_tag"], d.dev_off, P.TALP_GPU_SORTED_BY_START)
            batches.append((b, keep, d))
        torch.cuda.synchronize()
        e0.record(stream)
        for b, _, d in batches:
            P.talp_gpu_ingest_events(ctx.ctx, [b], stream)
            P.talp_gpu_region_metrics_device(ctx.ctx, [d.trace_id + (1 << 40)], P.TALP_GPU_ALL_REGIONS,
                                             out_dev.data_ptr(), stream)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms += e0.elapsed_time(e1)
        if wi == check_wave:
            # every trace of this wave against the oracle: the generated
            # records (the input the plan reduced) copied out, every unit
            # reduced by the oracle on the host cores, the metrics formed
            # from the oracle's own sums
            c0 = time.perf_counter()
            q = 0
            for d in dts:
                first = np.concatenate([[0], np.cumsum(d.devices_per_rank.astype(np.int64))])

                def fetch(r0, r1, d=d, first=first):
                    g0, g1 = int(first[r0]), int(first[r1])
                    x, y = int(d.dev_off[g0]), int(d.dev_off[g1])
                    return (d.dev_se[x:y].cpu().numpy(), d.dev_tag[x:y].cpu().numpy(),
                            np.asarray(d.dev_off[g0:g1 + 1], np.uint64) - np.uint64(x))

                du = oracle.device_unions_by_rank(fetch, d.n_ranks, d.devices_per_rank, d.region_window)
                ht = SimpleNamespace(n_ranks=d.n_ranks, region_window=d.region_window,
                                     host_se=d.host_se.cpu().numpy(), host_state=d.host_state.cpu().numpy(),
                                     host_off=np.asarray(d.host_off, np.uint64))
                for r in range(d.n_regions):
                    ref = oracle.metrics_from_sums(d.n_ranks, d.devices_per_rank, oracle.host_sums(ht, r), du[r],
                                                   d.region_window[r])
                    got = res[q + r]
                    for f in oracle.INT_FIELDS + oracle.RATIO_FIELDS:
                        exact &= got[f] == ref[f]
                q += d.n_regions
                whole_rec += d.n_records
            whole_traces = len(dts)
            whole_s = time.perf_counter() - c0
        # the smallest trace of the wave against the oracle (when it is small
        # enough for the host: waves of a few huge traces are not sampled)
        k = int(np.argmin([sp.n_records for sp in w]))
        if w[k].n_records <= 4_000_000:
            ht = igen.host_trace(w[k], igen.rank_ends(w[k]))
            q = sum(sp.n_regions for sp in w[:k])
            c0 = time.perf_counter()
            ref = [oracle.region_metrics(ht, r) for r in range(ht.n_regions)]
            cpu_s += time.perf_counter() - c0
            cpu_rec += ht.n_records
            for r in range(ht.n_regions):
                got = res[q + r]
                for f in oracle.INT_FIELDS + oracle.RATIO_FIELDS:
                    exact &= got[f] == ref[r][f]
            checked.append(int(w[k].trace_id))
        print(f"wave {wi + 1}/{len(wv)}: {info['records']} records, plan {plan_ms:.1f} ms, "
              f"plain {plain_ms:.1f} ms, {time.perf_counter() - g0:.1f} s", file=sys.stderr, flush=True)
        tot_rec += info["records"]
        tot_seg += info["segments"]
        plan.close()
        ctx.reset()
        del dts, arrays, batches
        torch.cuda.empty_cache()
    ck = clocks.stop()
    ctx.close()
    peak, peak_kind = measured_peaks()
    value = tot_rec / (plan_ms / 1000.0)
    achieved = BYTES_PER_RECORD * tot_rec / (plan_ms / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": len(wv), "warmup": len(wv),
        "ms_per_step": plan_ms / len(wv), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic (counter-based generator, made in HBM; the paper's traces are not available)",
        "config": {"workload": f"batched at full laws: {a.traces} traces, ranks log-uniform 1-512, 1-8 GPUs per rank, "
                               f"1e3-{ev_hi:g} device events per GPU log-uniform, 8 nested regions each",
                   "form": "per wave of whole traces: one CUDA-graph launch of a plan (a step = one wave; "
                           "warm-up launches for >= 150 ms, the mean of 3 timed launches)",
                   "waves": len(wv), "records": tot_rec, "bytes": BYTES_PER_RECORD * tot_rec, "segments": tot_seg,
                   "wave_records_max": int(a.wave_records), "generate_s": gen_s, "plan_build_s": build_s,
                   "plain_one_trace_per_launch_events_per_s": tot_rec / (plain_ms / 1000.0),
                   "batched_over_plain": plain_ms / plan_ms,
                   "oracle_checked_traces": checked, "bit_exact_sampled_vs_oracle": bool(exact),
                   "oracle_whole_wave": {"wave": check_wave, "traces": whole_traces, "records": whole_rec,
                                         "oracle_s": round(whole_s, 1),
                                         "what": "every unit and every metric field of every trace of the wave"},
                   "l2": "every wave far larger than L2; no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "whole graph (prep, sweep, fixup, finalize), summed over waves",
                     "kernel_ms": plan_ms, "peak_source": f"{peak_kind} hbm_gbs"},
        "cpu_baseline": {"value": cpu_rec / cpu_s if cpu_s else None, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"the smallest trace of every wave ({cpu_rec} records), {cpu_s:.2f} s"},
        "e2e": None, "gpu_launches": launches, "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    return 0 if exact else 1


def run_concurrency(a):
    line = measure_concurrency(a)
    print(json.dumps(line), flush=True)
    return 0 if line["config"]["bit_exact_rank0_vs_oracle"] else 1


def measure_concurrency(a, t=None):
    """Concurrency profile (time with >= k active records per device, k =
    1..8, all kinds and kernels only) of the plain large trace's devices, one
    call per step through the C ABI with the records resident in HBM (`t`:
    the trace, when the caller has generated it already)."""
    import torch
    import oracle
    import paper_2603_26576_b300 as P
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    if t is None:
        t = tg.plain_large(scale=a.scale)
    arr = dict(host_se=torch.from_numpy(t.host_se).to(dev), host_state=torch.from_numpy(t.host_state).to(dev),
               dev_se=torch.from_numpy(t.dev_se).to(dev), dev_tag=torch.from_numpy(t.dev_tag).to(dev))
    b, keep = P.batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, arr["host_se"],
                                  arr["host_state"], t.host_off, arr["dev_se"], arr["dev_tag"], t.dev_off)
    ctx = P.Context(0)
    stream = torch.cuda.Stream()
    region = 0
    clocks = Clocks(0)
    clocks.start()
    warm_until(lambda: P.talp_gpu_concurrency(ctx.ctx, b, region, stream), max(a.warmup, 3))
    res = P.talp_gpu_concurrency(ctx.ctx, b, region, stream)
    P.talp_gpu_profile_read(ctx.ctx)
    l0 = P.talp_gpu_profile_read(ctx.ctx)["kernel_launches"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(a.steps):
        P.talp_gpu_concurrency(ctx.ctx, b, region, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    launches = P.talp_gpu_profile_read(ctx.ctx)["kernel_launches"] - l0
    N = t.n_dev
    # parity on one rank's devices against the oracle
    from paper_2603_26576_b300 import shard
    s0 = shard.shard_of(t, [0])
    c0 = time.perf_counter()
    want = oracle.concurrency(s0, region, P.TALP_GPU_CONC_LEVELS)
    cpu_s = time.perf_counter() - c0
    exact = bool(np.array_equal(res[: int(s0.devices_per_rank.sum())], want))
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_RECORD * N / (ms / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": N / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic (seeded generator; the paper's traces are not available)",
        "config": {"workload": "concurrency profile of the plain large trace's 256 devices (2M events each, "
                               "4 streams), levels 1-8, all records and kernels only, region 0"
                               + ("" if a.scale == 1.0 else f" (scale {a.scale})"),
                   "records_per_step": N, "form": "talp_gpu_concurrency, one synchronous call per step",
                   "l2": "records (%.1f GB) larger than L2; no flush" % (BYTES_PER_RECORD * N / 1e9),
                   "bit_exact_rank0_vs_oracle": exact},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None,
                     "kernel": "main levels pass + per-device chunk scan + fix-up of chunks' leading tiles (every "
                               "record read once; the fix-up rereads a few tiles)",
                     "kernel_ms": ms, "peak_source": f"{peak_kind} hbm_gbs"},
        "cpu_baseline": {"value": s0.n_records / cpu_s if cpu_s else None, "unit": UNIT, "cores": 1,
                         "kind": "oracle", "sample": f"rank 0's 4 devices ({int(s0.dev_se.shape[0])} records), "
                                                     f"{cpu_s:.2f} s"},
        "e2e": None, "gpu_launches": launches, "clocks": ck,
    }
    ctx.close()
    del arr, b, keep
    torch.cuda.empty_cache()
    return line


def run_raw(a):
    line = measure_raw(a)
    print(json.dumps(line), flush=True)
    return 0 if line["config"]["bit_exact_raw_vs_lanes"] else 1


def measure_raw(a):
    """Raw activity records: the plain trace's device records as per-rank
    delivery buffers (all devices and streams interleaved in completion
    order), ingested through talp_gpu_ingest_raw from HBM and reduced, one
    synchronous step per call; against the same records already in lanes
    in start order."""
    import torch
    import oracle
    import paper_2603_26576_b300 as P
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    scale = a.scale if a.scale != 1.0 else 0.25
    t = tg.plain_large(scale=scale)
    r = tg.to_raw(t)
    up = lambda x: torch.from_numpy(x).to(dev)  # noqa: E731
    arr = dict(host_se=up(t.host_se), host_state=up(t.host_state), raw_se=up(r.raw_se), raw_tag=up(r.raw_tag),
               raw_dev=up(r.raw_dev))
    lanes = dict(host_se=arr["host_se"], host_state=arr["host_state"], dev_se=up(t.dev_se), dev_tag=up(t.dev_tag))
    rb, keep = P.raw_batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, arr["host_se"],
                                       arr["host_state"], t.host_off, arr["raw_se"], arr["raw_tag"], arr["raw_dev"],
                                       r.raw_off)
    lb, keep2 = P.batch_from_arrays(t.trace_id + 1, t.devices_per_rank, t.region_window, lanes["host_se"],
                                    lanes["host_state"], t.host_off, lanes["dev_se"], lanes["dev_tag"], t.dev_off,
                                    P.TALP_GPU_SORTED_BY_START)
    ctx = P.Context(0)
    stream = torch.cuda.Stream()
    R = t.n_regions
    out_dev = torch.empty(R * 200, dtype=torch.uint8, device=dev)
    hold = max(1, a.hold_calls)
    hold_batches = []
    if hold > 1:
        # the same records as `hold` delivery buffers: all but the last with
        # hold-back, the last one flushes; the first one starts the trace
        for j, p in enumerate(tg.raw_deliveries(r, hold, seed=5)):
            pa = [up(p.trace.host_se), up(p.trace.host_state), up(p.raw_se), up(p.raw_tag), up(p.raw_dev)]
            fl = (P.TALP_GPU_HOLD_BACK if j < hold - 1 else 0) | (P.TALP_GPU_APPEND if j else 0)
            hold_batches.append(P.raw_batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, pa[0],
                                                        pa[1], p.trace.host_off, pa[2], pa[3], pa[4], p.raw_off,
                                                        fl, p.stream_mask) + (pa,))

    def step_raw():
        if hold > 1:
            for hb_, _, _ in hold_batches:
                P.talp_gpu_ingest_raw(ctx.ctx, [hb_], stream)
        else:
            P.talp_gpu_ingest_raw(ctx.ctx, [rb], stream)
        P.talp_gpu_region_metrics_device(ctx.ctx, [t.trace_id], P.TALP_GPU_ALL_REGIONS, out_dev.data_ptr(), stream)

    def step_lanes():
        P.talp_gpu_ingest_events(ctx.ctx, [lb], stream)
        P.talp_gpu_region_metrics_device(ctx.ctx, [t.trace_id + 1], P.TALP_GPU_ALL_REGIONS, out_dev.data_ptr(),
                                         stream)

    def timed(fn, k):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    clocks = Clocks(0)
    clocks.start()
    warm_until(step_raw, max(a.warmup, 3))
    P.talp_gpu_profile_read(ctx.ctx)
    l0 = P.talp_gpu_profile_read(ctx.ctx)["kernel_launches"]
    ms = timed(step_raw, a.steps)
    ck = clocks.stop()
    launches = P.talp_gpu_profile_read(ctx.ctx)["kernel_launches"] - l0 + a.steps
    warm_until(step_lanes, max(a.warmup, 3), 0.3)
    ms_lanes = timed(step_lanes, a.steps)
    got = P.talp_gpu_region_metrics(ctx.ctx, t.trace_id, P.TALP_GPU_ALL_REGIONS, stream, n_regions=R)
    lane_res = P.talp_gpu_region_metrics(ctx.ctx, t.trace_id + 1, P.TALP_GPU_ALL_REGIONS, stream, n_regions=R)
    same = all(P.metrics_to_dict(x) == dict(P.metrics_to_dict(y), trace_id=t.trace_id) for x, y in zip(got, lane_res))
    N = t.n_records
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_RECORD * N / (ms / 1000.0) / 1e9
    c0 = time.perf_counter()
    oracle.region_metrics(tg.plain_large(scale=scale, n_ranks=1), 0)
    cpu_s = time.perf_counter() - c0
    line = {
        "metric": METRIC, "value": N / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic (seeded generator; the paper's traces are not available)",
        "config": {"workload": f"plain large trace at scale {scale:g} as raw per-rank delivery buffers (4 devices x "
                               "4 streams per rank interleaved in completion order)",
                   "records_per_step": N,
                   "form": ("talp_gpu_ingest_raw + metrics, one synchronous call per step" if hold == 1 else
                            f"{hold} delivery buffers per step through talp_gpu_ingest_raw with hold-back "
                            "(the last one flushes), then metrics"),
                   "lanes_in_start_order_ms_per_step": ms_lanes, "raw_over_lanes_time": ms / ms_lanes,
                   "bit_exact_raw_vs_lanes": same,
                   "l2": "records (%.1f GB) larger than L2; no flush" % (BYTES_PER_RECORD * N / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "whole step (scatter, sweep, merge sort, re-sweep, finalize)",
                     "kernel_ms": ms, "peak_source": f"{peak_kind} hbm_gbs"},
        "cpu_baseline": {"value": None if not cpu_s else (N / t.n_ranks) / cpu_s, "unit": UNIT, "cores": 1,
                         "kind": "oracle", "sample": f"one rank of the workload, {cpu_s:.2f} s"},
        "e2e": None, "gpu_launches": launches, "clocks": ck,
    }
    ctx.close()
    del arr, lanes, rb, keep, lb, keep2, hold_batches
    torch.cuda.empty_cache()
    return line


def run_threads(a):
    """Host tree with threads: the plain large trace with 8 threads per rank
    (one host unit per thread; 64 processes x 8 threads x 4 GPUs), ingested
    from HBM and reduced to the thread tree of every region, one synchronous
    step per call; against the same step with the paper's tree."""
    import torch
    import oracle
    import paper_2603_26576_b300 as P
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    t = tg.threaded_large(scale=a.scale)
    po = t.meta["proc_off"]
    up = lambda x: torch.from_numpy(x).to(dev)  # noqa: E731
    arr = dict(host_se=up(t.host_se), host_state=up(t.host_state), dev_se=up(t.dev_se), dev_tag=up(t.dev_tag))
    b, keep = P.batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, arr["host_se"],
                                  arr["host_state"], t.host_off, arr["dev_se"], arr["dev_tag"], t.dev_off,
                                  P.TALP_GPU_SORTED_BY_START)
    ctx = P.Context(0)
    stream = torch.cuda.Stream()
    R = t.n_regions
    out_dev = torch.empty(R * 200, dtype=torch.uint8, device=dev)

    out_thr = torch.empty(R * 112, dtype=torch.uint8, device=dev)

    def step_threads():
        P.talp_gpu_ingest_events(ctx.ctx, [b], stream)
        P.talp_gpu_thread_metrics_device(ctx.ctx, t.trace_id, P.TALP_GPU_ALL_REGIONS, po, out_thr.data_ptr(), stream)

    def step_paper():
        P.talp_gpu_ingest_events(ctx.ctx, [b], stream)
        P.talp_gpu_region_metrics_device(ctx.ctx, [t.trace_id], P.TALP_GPU_ALL_REGIONS, out_dev.data_ptr(), stream)

    def timed(fn, k):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    clocks = Clocks(0)
    clocks.start()
    warm_until(step_paper, max(a.warmup, 3), 0.3)
    warm_until(step_threads, max(a.warmup, 3))
    P.talp_gpu_profile_read(ctx.ctx)
    l0 = P.talp_gpu_profile_read(ctx.ctx)["kernel_launches"]
    ms = timed(step_threads, a.steps)
    ck = clocks.stop()
    launches = P.talp_gpu_profile_read(ctx.ctx)["kernel_launches"] - l0
    ms_paper = timed(step_paper, a.steps)
    step_threads()
    torch.cuda.synchronize()
    got = P.thread_tree_from_bytes(out_thr.cpu().numpy().tobytes())
    exact = got == P.talp_gpu_thread_metrics(ctx.ctx, t.trace_id, P.TALP_GPU_ALL_REGIONS, po, stream,
                                             n_regions=R) and all(g == dict(oracle.thread_metrics(t, r, po), trace_id=t.trace_id, region=r)
                for r, g in enumerate(got))
    N = t.n_records
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_RECORD * N / (ms / 1000.0) / 1e9
    one = tg.add_threads(tg.plain_large(scale=a.scale, n_ranks=1), 8)
    c0 = time.perf_counter()
    for r in range(R):
        oracle.region_metrics(one, r)
        oracle.thread_metrics(one, r, one.meta["proc_off"])
    cpu_s = time.perf_counter() - c0
    line = {
        "metric": METRIC, "value": N / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic (seeded generator; the paper's traces are not available)",
        "config": {"workload": "plain large trace with 8 threads per rank (64 processes x 8 threads x 4 GPUs x "
                               "4 streams; 1 master + 7 fork-join workers)"
                               + ("" if a.scale == 1.0 else f" (scale {a.scale})"),
                   "records_per_step": N, "host_records": t.n_host,
                   "form": "talp_gpu_ingest_events (device records, start order) + "
                           "talp_gpu_thread_metrics_device of the 4 regions, stream-ordered",
                   "paper_tree_ms_per_step": ms_paper, "bit_exact_vs_oracle": exact,
                   "threads_over_paper_time": ms / ms_paper,
                   "l2": "records (%.1f GB) larger than L2; no flush" % (BYTES_PER_RECORD * N / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "whole step (sweep, fix-up, thread tree)",
                     "kernel_ms": ms, "peak_source": f"{peak_kind} hbm_gbs"},
        "cpu_baseline": {"value": None if not cpu_s else one.n_records / cpu_s, "unit": UNIT, "cores": 1,
                         "kind": "oracle", "sample": f"one process of the workload (8 threads, 4 GPUs): device "
                                                     f"unions, host sums and both trees of the 4 regions, "
                                                     f"{cpu_s:.2f} s"},
        "e2e": None, "gpu_launches": launches, "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0 if exact else 1


# ----------------------------------------------------------------- serving


class ServeLoad:
    """Client load of the serving workload: submitter threads with Poisson
    arrivals (or closed loop), and query threads asking every job for all
    its regions once per query period.  `api` is the served form or the
    plain form behind the same two calls."""

    def __init__(self, jobs, submit, query, rate, query_s, n_sub=8, n_q=16, seed=7):
        self.jobs, self.submit, self.query = jobs, submit, query
        self.rate, self.query_s = rate, query_s
        self.n_sub, self.n_q, self.seed = n_sub, n_q, seed
        self.next_q = [0] * len(jobs)
        self.sub_records = 0
        self.lat = []
        self.errors = []

    def run(self, seconds, closed_loop=False):
        stop = threading.Event()
        self.lat = []
        t_start = time.perf_counter()

        def submitter(tid):
            rng = np.random.default_rng([self.seed, tid, len(self.lat), int(t_start * 1e3) & 0xFFFF])
            mine = list(range(tid, len(self.jobs), self.n_sub))
            t_next = time.perf_counter()
            k = 0
            try:
                while not stop.is_set():
                    if closed_loop:
                        j = mine[k % len(mine)]
                        k += 1
                    else:
                        t_next += rng.exponential(self.n_sub / self.rate)
                        d = t_next - time.perf_counter()
                        if d > 0:
                            time.sleep(d)
                        j = mine[int(rng.integers(0, len(mine)))]
                    b = self.jobs[j].batch(self.next_q[j])
                    self.submit(j, b)
                    self.next_q[j] += 1
                    self.sub_records += b.n_records
            except Exception as e:  # reported in the result line
                self.errors.append(repr(e))

        def querier(tid):
            mine = list(range(tid, len(self.jobs), self.n_q))
            t_tick = time.perf_counter()
            lat = []
            try:
                while not stop.is_set():
                    for j in mine:
                        q0 = time.perf_counter()
                        self.query(j)
                        lat.append(time.perf_counter() - q0)
                    t_tick += self.query_s
                    d = t_tick - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    else:
                        t_tick = time.perf_counter()
            except Exception as e:
                self.errors.append(repr(e))
            self.lat.extend(lat)

        th = [threading.Thread(target=submitter, args=(i,)) for i in range(self.n_sub)]
        th += [threading.Thread(target=querier, args=(i,)) for i in range(self.n_q)]
        for x in th:
            x.start()
        time.sleep(seconds)
        stop.set()
        for x in th:
            x.join()
        return time.perf_counter() - t_start


def _pct(v, p):
    if not v:
        return None
    v = sorted(v)
    return v[min(len(v), max(1, int(np.ceil(p * len(v))))) - 1]


def run_serving(a):
    line = measure_serving(a)
    print(json.dumps(line), flush=True)
    return 0 if line["bit_exact_sampled_jobs"]["exact"] and not line["errors"] else 1


def measure_serving(a):
    """Served form: many jobs stream batches into device-resident state while
    clients query it; against the plain form (one ingest per batch, one
    synchronous metrics call per query) at the same load."""
    import torch
    import oracle
    import paper_2603_26576_b300 as P
    sys.setswitchinterval(0.0002)
    torch.cuda.set_device(0)
    t0 = time.time()
    jobs = tg.serving_jobs(n_jobs=a.jobs)
    gen_s = time.time() - t0
    R = jobs[0].n_regions
    step_s = a.step_s
    paced_s = (a.warmup + a.steps) * step_s
    # region windows cover what the paced phases deliver (later batches are clipped)
    horizon = int(a.rate / a.jobs * (paced_s + a.plain_s + a.native_s) * 2 + 64)
    wins = [j.windows(horizon) for j in jobs]
    max_rec = max(b.n_records for j in jobs for b in j.batches)

    ctx = P.Context(0)
    srv = P.Server(ctx, max_jobs=a.jobs, max_slice_records=max_rec, staging_slices=128)
    for j, w in zip(jobs, wins):
        srv.open_job(j.job_id, j.trace.devices_per_rank, w)

    def s_submit(k, b):
        srv.submit(k, b.host_se, b.host_state, b.host_off, b.dev_se, b.dev_tag, b.dev_off)

    lib = P.load_library()

    def s_query(k):
        o = (P.talp_gpu_metrics * R)()
        st = lib.talp_gpu_server_query(srv.handle, k, P.TALP_GPU_ALL_REGIONS, o)
        if st != 0:
            raise P.TalpGpuError(st, P.talp_gpu_last_error())

    load = ServeLoad(jobs, s_submit, s_query, a.rate, a.query_ms / 1000.0)
    # warm-up phase, then the timed phase (paced arrivals)
    load.run(a.warmup * step_s)
    srv.drain()
    P.talp_gpu_profile(ctx.ctx, True)
    P.talp_gpu_profile_read(ctx.ctx)
    l0 = P.talp_gpu_profile_read(ctx.ctx)["kernel_launches"]
    s0 = srv.stats()
    clocks = Clocks(0)
    clocks.start()
    time.sleep(0.2)
    s0 = srv.stats()
    wall = load.run(a.steps * step_s)
    s1 = srv.stats()
    ck = clocks.stop()
    lat_paced = list(load.lat)
    srv.drain()
    prof = P.talp_gpu_profile_read(ctx.ctx)
    P.talp_gpu_profile(ctx.ctx, False)
    s2 = srv.stats()
    folded = s1["records_folded"] - s0["records_folded"]
    value = folded / wall
    launches = (prof["kernel_launches"] - l0) + (s2["query_batches"] - s0["query_batches"])
    waves = s2["waves"] - s0["waves"]
    n_queries = s2["queries"] - s0["queries"]
    sub_slices = s2["slices_submitted"] - s0["slices_submitted"]
    # the same paced load from native client threads: the query latency an
    # application sees when it calls the library from its own threads
    native = None
    if a.native_s > 0:
        from tracegen import serve_load
        keep_nat, njobs = [], []
        for k, j in enumerate(jobs):
            assert j.job_id == k
            arr = (P.talp_gpu_trace_batch * len(j.batches))()
            for i, sb in enumerate(j.batches):
                b, kp = P.batch_from_arrays(j.job_id, np.zeros(0, np.uint32), np.zeros((0, 0, 2), np.int64),
                                            sb.host_se, sb.host_state, sb.host_off, sb.dev_se, sb.dev_tag,
                                            sb.dev_off, P.TALP_GPU_SORTED_BY_START if sb.sorted_by_start else 0)
                arr[i] = b
                keep_nat.append(kp)
            keep_nat.append(arr)
            njobs.append(dict(job_id=j.job_id, n_ranks=int(j.trace.n_ranks), n_devices=int(j.trace.m_devices),
                              n_slices=len(j.batches), n_regions=R, span=int(j.span),
                              slices=ctypes.addressof(arr)))
        fn = lambda f: ctypes.cast(f, ctypes.c_void_p).value  # noqa: E731
        na0 = srv.stats()
        nr = serve_load.run(srv.handle, fn(lib.talp_gpu_server_submit), fn(lib.talp_gpu_server_query), njobs,
                            load.next_q, a.rate, a.query_ms / 1000.0, a.native_s)
        na1 = srv.stats()
        del keep_nat
        native = {"p50": 1000.0 * _pct(nr["lat"], 0.5) if nr["lat"] else None,
                  "p99": 1000.0 * _pct(nr["lat"], 0.99) if nr["lat"] else None,
                  "max": 1000.0 * max(nr["lat"]) if nr["lat"] else None, "queries": nr["queries"],
                  "queries_per_s": nr["queries"] / nr["wall_s"],
                  "batches_per_s": nr["slices"] / nr["wall_s"],
                  "events_per_s": (na1["records_folded"] - na0["records_folded"]) / nr["wall_s"],
                  "seconds": nr["wall_s"], "errors": nr["errors"], "first_error": nr["first_error"],
                  "measured": "native client threads (8 submitters, 16 queriers) calling the C ABI; "
                              "around each talp_gpu_server_query call"}
    # saturation: closed-loop submitters, queries still every period
    sa0 = srv.stats()
    sat_wall = load.run(a.sat_s, closed_loop=True) if a.sat_s > 0 else 0.0
    sa1 = srv.stats()
    lat_sat = list(load.lat) if a.sat_s > 0 else []
    srv.drain()
    # bit-exact check of sampled jobs against the oracle on what they received
    order = sorted(range(len(jobs)), key=lambda k: sum(jobs[k].batch(q).n_records for q in range(load.next_q[k])))
    sample = order[:3]
    exact = True
    cpu_records, cpu_s = 0, 0.0
    for k in sample:
        got = srv.query(k)
        pt = jobs[k].prefix(load.next_q[k], wins[k])
        c0 = time.perf_counter()
        ref = [oracle.region_metrics(pt, r) for r in range(R)]
        cpu_s += time.perf_counter() - c0
        cpu_records += pt.n_records
        for r in range(R):
            for f in P._lib.INT_FIELDS + P._lib.RATIO_FIELDS:
                if got[r][f] != ref[r][f]:
                    exact = False
    st_native = srv.stats()
    srv.close()
    ctx.close()

    # ---- plain form at the same load: one ingest per batch, one synchronous
    # metrics call per query, serialised on one context
    ctx2 = P.Context(0)
    lock = threading.Lock()
    stream = torch.cuda.Stream()
    for j, w in zip(jobs, wins):
        t = j.trace
        e = tg.Slice(np.zeros((0, 2), np.int64), np.zeros(0, np.uint8), np.zeros(t.n_ranks + 1, np.uint64),
                     np.zeros((0, 2), np.int64), np.zeros(0, np.uint8), np.zeros(t.m_devices + 1, np.uint64))
        b, keep = P.batch_from_arrays(j.job_id, t.devices_per_rank, w, e.host_se, e.host_state, e.host_off,
                                      e.dev_se, e.dev_tag, e.dev_off, P.TALP_GPU_SORTED_BY_START)
        P.talp_gpu_ingest_events(ctx2.ctx, [b], stream)

    def p_submit(k, b):
        t = jobs[k].trace
        bb, keep = P.batch_from_arrays(k, t.devices_per_rank, wins[k], b.host_se, b.host_state, b.host_off,
                                       b.dev_se, b.dev_tag, b.dev_off,
                                       P.TALP_GPU_SORTED_BY_START | P.TALP_GPU_APPEND)
        with lock:
            P.talp_gpu_ingest_events(ctx2.ctx, [bb], stream)
        del keep

    def p_query(k):
        with lock:
            P.talp_gpu_region_metrics(ctx2.ctx, k, P.TALP_GPU_ALL_REGIONS, stream, n_regions=R)

    pload = ServeLoad(jobs, p_submit, p_query, a.rate, a.query_ms / 1000.0)
    pload.next_q = [0] * len(jobs)
    pr0 = pload.sub_records
    clocks_p = Clocks(0)
    clocks_p.start()
    p_wall = pload.run(a.plain_s)
    torch.cuda.synchronize()
    ck_plain = clocks_p.stop()
    p_rec = pload.sub_records - pr0
    lat_plain = list(pload.lat)
    # the plain form's sampled jobs against the oracle on what they received
    p_order = sorted(range(len(jobs)), key=lambda k: sum(jobs[k].batch(q).n_records for q in range(pload.next_q[k])))
    p_sample = p_order[:3]
    p_exact = True
    for k in p_sample:
        got = [P.metrics_to_dict(x) for x in
               P.talp_gpu_region_metrics(ctx2.ctx, k, P.TALP_GPU_ALL_REGIONS, stream, n_regions=R)]
        pt = jobs[k].prefix(pload.next_q[k], wins[k])
        ref = [oracle.region_metrics(pt, r) for r in range(R)]
        for r in range(R):
            for f in P._lib.INT_FIELDS + P._lib.RATIO_FIELDS:
                if got[r][f] != ref[r][f]:
                    p_exact = False
    ctx2.close()

    peak, peak_kind = measured_peaks()
    sweep_ms = prof["sweep_ms"] / max(1, prof["sweep_launches"])
    rec_per_sweep = prof["sweep_records"] / max(1, prof["sweep_launches"])
    achieved = BYTES_PER_RECORD * rec_per_sweep / (sweep_ms / 1000.0) / 1e9 if sweep_ms > 0 else 0.0
    ms = lambda x: None if x is None else 1000.0 * x  # noqa: E731
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1000.0 * wall / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic (seeded generator; the paper's traces are not available)",
        "config": {"workload": f"serving: {a.jobs} jobs (8-256 ranks x 1-4 GPUs), batches of 1k-100k events "
                               f"log-uniform, Poisson {a.rate:g} batches/s, a query per job every "
                               f"{a.query_ms:g} ms (all {R} nested regions)",
                   "step": f"{step_s:g} s of served load (wall clock)", "generate_s": gen_s,
                   "l2": "each batch crosses PCIe once; device state is small and stays resident"},
        "latency_ms": {"p50": ms(_pct(lat_paced, 0.5)), "p99": ms(_pct(lat_paced, 0.99)),
                       "max": ms(max(lat_paced) if lat_paced else None), "queries": len(lat_paced),
                       "measured": "client side, around each query call"},
        "native_client_latency_ms": native,
        "server_latency_ms": {"p50": st_native["query_p50_ms"], "p99": st_native["query_p99_ms"],
                              "max": st_native["query_max_ms"],
                              "measured": "inside the library, whole run"},
        "served": {"queries_per_s": n_queries / wall, "batches_per_s": sub_slices / wall,
                   "waves_per_s": waves / wall, "query_batches": s2["query_batches"] - s0["query_batches"]},
        "saturation": None if not sat_wall else {
            "events_per_s": (sa1["records_folded"] - sa0["records_folded"]) / sat_wall,
            "batches_per_s": (sa1["slices_folded"] - sa0["slices_folded"]) / sat_wall,
            "p50_ms": ms(_pct(lat_sat, 0.5)), "p99_ms": ms(_pct(lat_sat, 0.99)), "queries": len(lat_sat)},
        "plain_same_load": {"events_per_s": p_rec / p_wall, "queries_per_s": len(lat_plain) / p_wall,
                            "p50_ms": ms(_pct(lat_plain, 0.5)), "p99_ms": ms(_pct(lat_plain, 0.99)),
                            "form": "one APPEND ingest per batch + one synchronous metrics call per query",
                            "bit_exact_sampled_jobs": {"jobs": p_sample, "exact": p_exact}},
        "bit_exact_sampled_jobs": {"jobs": sample, "exact": exact},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None, "traffic": None, "kernel": "talp::sweep_kernel",
                     "kernel_ms": sweep_ms, "records_per_launch": rec_per_sweep,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "note": "small waves: the sweep is latency-bound, not bandwidth-bound"},
        "cpu_baseline": {"value": cpu_records / cpu_s if cpu_s else None, "unit": UNIT, "cores": 1,
                         "kind": "oracle", "sample": f"{len(sample)} smallest jobs' received streams "
                                                     f"({cpu_records} records), {cpu_s:.1f} s"},
        "e2e": {"value": value, "unit": UNIT,
                "h2d_bytes_per_step": int(BYTES_PER_RECORD * folded / a.steps),
                "d2h_bytes_per_step": int(n_queries * R * 184 / a.steps),
                "note": "the served form takes host buffers: value is already end to end"},
        "gpu_launches": launches, "clocks": ck, "clocks_plain": ck_plain, "errors": load.errors + pload.errors + (
            [f"native client: {native['errors']} failed calls, first status {native['first_error']}"]
            if native and native["errors"] else []),
    }
    return line


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "batched":
        return run_batched(a)
    if a.workload == "batched-full":
        return run_batched_full(a)
    if a.workload == "concurrency":
        return run_concurrency(a)
    if a.workload == "threads":
        return run_threads(a)
    if a.workload == "raw":
        return run_raw(a)
    if a.workload == "serving":
        return run_serving(a)
    import torch
    import paper_2603_26576_b300 as P

    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", local)

    t, _ = workload(a.workload, a.scale, rank)
    if a.workload == "scale":
        # generated straight into HBM by the generator's device twin
        from tracegen import igen
        (t,) = igen.generate_device([t], device=local)
        d_arrays = dict(host_se=t.host_se, host_state=t.host_state, dev_se=t.dev_se, dev_tag=t.dev_tag)
    else:
        if a.unsorted:
            t = tg.split_runs(t, a.runs, seed=1) if a.runs > 0 else tg.interleave_lanes(t)
        # device-resident copies of the records
        d_arrays = dict(host_se=torch.from_numpy(t.host_se).to(dev),
                        host_state=torch.from_numpy(t.host_state).to(dev),
                        dev_se=torch.from_numpy(t.dev_se).to(dev), dev_tag=torch.from_numpy(t.dev_tag).to(dev))
    N = t.n_records
    R = t.n_regions
    torch.cuda.synchronize()
    ctx = P.Context(local)
    stream = torch.cuda.Stream(device=dev)
    if a.unsorted:
        flags = P.TALP_GPU_GROUPED_BY_STREAM if a.grouped_hint else (P.TALP_GPU_NOT_SORTED if a.not_sorted_hint else 0)
    else:
        flags = P.TALP_GPU_SORTED_BY_START
    batch_d, keep_d = P.batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, d_arrays["host_se"],
                                          d_arrays["host_state"], t.host_off, d_arrays["dev_se"],
                                          d_arrays["dev_tag"], t.dev_off, flags)
    out_dev = torch.empty(R * 200, dtype=torch.uint8, device=dev)

    def step_device():
        P.talp_gpu_ingest_events(ctx.ctx, [batch_d], stream)
        P.talp_gpu_region_metrics_device(ctx.ctx, [t.trace_id], P.TALP_GPU_ALL_REGIONS, out_dev.data_ptr(), stream)

    clocks = Clocks(torch.cuda.current_device() if ws == 1 else local)
    clocks.start()
    warm_until(step_device, max(a.warmup, 3))
    # the results of the warm-up are checked once through the host API
    res = P.talp_gpu_region_metrics(ctx.ctx, t.trace_id, P.TALP_GPU_ALL_REGIONS, stream, n_regions=R)
    step_device()                      # one more untimed step after the host-side check
    P.talp_gpu_profile(ctx.ctx, True)
    P.talp_gpu_profile_read(ctx.ctx)
    launches0 = P.talp_gpu_profile_read(ctx.ctx)["kernel_launches"]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    ev[0].record(stream)
    for q in range(a.steps):
        step_device()
        ev[q + 1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = ev[0].elapsed_time(ev[-1])
    per_step = sorted(ev[q].elapsed_time(ev[q + 1]) for q in range(a.steps))
    prof = P.talp_gpu_profile_read(ctx.ctx)
    P.talp_gpu_profile(ctx.ctx, False)
    launches = prof["kernel_launches"] - launches0
    if ws > 1:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    value = N * a.steps * ws / (ms / 1000.0)

    # ---- end to end through the C ABI from pinned host buffers
    e2e = None
    if not a.no_e2e:
        def pinned(x):
            if hasattr(x, "is_cuda"):
                h = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
                h.copy_(x)
                return h
            return torch.from_numpy(x).pin_memory()
        h_arrays = {k: pinned(getattr(t, k)) for k in ("host_se", "host_state", "dev_se", "dev_tag")}
        batch_h, keep_h = P.batch_from_arrays(t.trace_id, t.devices_per_rank, t.region_window, h_arrays["host_se"],
                                              h_arrays["host_state"], t.host_off, h_arrays["dev_se"],
                                              h_arrays["dev_tag"], t.dev_off, flags)

        def step_e2e():
            P.talp_gpu_ingest_events(ctx.ctx, [batch_h], stream)
            return P.talp_gpu_region_metrics(ctx.ctx, t.trace_id, P.TALP_GPU_ALL_REGIONS, stream, n_regions=R)

        step_e2e()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        k = max(1, a.e2e_steps)
        w0 = time.perf_counter()
        for _ in range(k):
            step_e2e()
        w1 = time.perf_counter()
        el = w1 - w0
        if ws > 1:
            tt = torch.tensor([el], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            el = float(tt.item())
        h2d = sum(int(v.numel() * v.element_size()) for v in h_arrays.values())
        meta = t.devices_per_rank.nbytes + t.region_window.nbytes + t.host_off.nbytes + t.dev_off.nbytes
        e2e = {"value": N * k * ws / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d + meta),
               "d2h_bytes_per_step": int(R * 200), "steps": k}

    # ---- roofline of the sweep kernel (records in start order), or of the
    # sort stage (device records out of order: the fused merge-sweep reads
    # every device record once, 17 B each)
    peak, peak_kind = measured_peaks()
    sweep_ms = prof["sweep_ms"] / max(1, prof["sweep_launches"])
    if a.unsorted:
        n_dev = int(t.dev_off[-1])
        sort_ms = prof["sort_ms"] / max(1, prof["sort_launches"])
        achieved = BYTES_PER_RECORD * n_dev / (sort_ms / 1000.0) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None,
                "kernel": "sort stage (run finding, talp::fms_kernel and its plan and fix-up kernels)",
                "kernel_ms": sort_ms, "records_per_launch": n_dev,
                "first_sweep_ms": sweep_ms, "peak_source": f"{peak_kind} hbm_gbs"}
    else:
        achieved = BYTES_PER_RECORD * N / (sweep_ms / 1000.0) / 1e9
        tpr = sweep_traffic_per_record() if a.workload == "plain" else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (tpr * N) if tpr is not None else None, "kernel": "talp::sweep_kernel",
                "kernel_ms": sweep_ms, "peak_source": f"{peak_kind} hbm_gbs"}

    # ---- CPU oracle on a bounded sample (rank 0, N = 1 only)
    cpu = cpu_all = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        s = oracle_sample(a.workload, a.scale)
        reps, tot = 0, 0.0
        while reps < 1 or (tot < 10.0 and reps < 20):   # about 10 s of CPU work
            tot += time_oracle(s)
            reps += 1
        dt = tot / reps
        cpu = {"value": s.n_records / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one rank of the workload ({s.m_devices} devices, {s.n_records} records) x "
                         f"{s.n_regions} regions, {reps} times: {tot:.1f} s", **host_cpu()}
        v_all, p_all, n_all = oracle_all_cores(a.workload, a.scale)
        cpu_all = {"value": v_all, "unit": UNIT, "cores": p_all, "kind": "oracle",
                   "sample": f"the same sample ({n_all} records) in {p_all} processes at once, one per core"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic (seeded generator; the paper's traces are not available)",
            "config": {"workload": workload_name(a), "records_per_step": N, "bytes_per_step": BYTES_PER_RECORD * N,
                       "regions": R, "l2": "inputs (%.1f GB) larger than L2; no flush" % (BYTES_PER_RECORD * N / 1e9),
                       "input_order": ((f"each device's records dealt into {a.runs} sorted runs laid end to end"
                                        if a.runs > 0 else "device records grouped by stream, each stream in start "
                                        "order") + ("; caller flag TALP_GPU_GROUPED_BY_STREAM: each device's runs "
                                                    "found from its stream ids, merged without a first sweep"
                                                    if a.grouped_hint else
                                                    "; caller hint TALP_GPU_NOT_SORTED: every device is sorted "
                                                    "without a first sweep" if a.not_sorted_hint else
                                                    "; the library finds the out-of-order devices and sorts them "
                                                    "(sort stage)"))
                       if a.unsorted else "device records in start order (caller asserts SORTED_BY_START)",
                       "kernel_overlap": "each device's 4 kernel streams are independent lanes: kernels of "
                                         "different streams overlap and are merged by the flattening",
                       "hbm_gb_per_s": BYTES_PER_RECORD * N * a.steps / (ms / 1000.0) / 1e9,
                       "ms_per_step_best": per_step[0], "ms_per_step_median": per_step[len(per_step) // 2]},
            "roofline": roof, "cpu_baseline": cpu, "cpu_all_cores": cpu_all, "e2e": e2e, "gpu_launches": launches,
            "clocks": ck,
            "check": {"elapsed_ns_region0": res[0].elapsed_ns, "dev_pe_region0": res[0].dev_pe},
        }
    ctx.close()
    rc = 0
    if rank == 0 and ws == 1 and a.workload == "plain" and not a.unsorted and a.scale == 1.0 and not a.no_extras:
        # the metric's latency half and the spec comparisons, measured
        # in the same run after the plain workload's buffers are released
        del d_arrays, batch_d, keep_d
        if e2e is not None:
            del h_arrays, batch_h, keep_h
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        extra = default_extras(a, t, res)
        rc = extra.pop("_rc")
        line.update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return rc


def measure_sort_stage(a, t, want):
    """The plain large trace `t` with each device's records grouped by stream
    (each stream in start order, as per-stream activity buffers deliver them):
    the library finds the devices out of order and sorts them (the sort
    stage: runs found by the first sweep, merged and swept in one pass by the
    fused merge-sweep).  Same step as the plain leg (ingest + metrics of every
    region); the results must equal `want`, the start-ordered run's."""
    import torch
    import paper_2603_26576_b300 as P
    dev = torch.device("cuda", 0)
    u = tg.interleave_lanes(t)
    arr = {k: torch.from_numpy(getattr(u, k)).to(dev) for k in ("host_se", "host_state", "dev_se", "dev_tag")}
    b, keep = P.batch_from_arrays(u.trace_id, u.devices_per_rank, u.region_window, arr["host_se"], arr["host_state"],
                                  u.host_off, arr["dev_se"], arr["dev_tag"], u.dev_off, 0)
    R = u.n_regions
    ctx = P.Context(0)
    stream = torch.cuda.Stream()
    out_dev = torch.empty(R * 200, dtype=torch.uint8, device=dev)

    def step():
        P.talp_gpu_ingest_events(ctx.ctx, [b], stream)
        P.talp_gpu_region_metrics_device(ctx.ctx, [u.trace_id], P.TALP_GPU_ALL_REGIONS, out_dev.data_ptr(), stream)

    clocks = Clocks(0)
    clocks.start()
    warm_until(step, 3)
    got = P.talp_gpu_region_metrics(ctx.ctx, u.trace_id, P.TALP_GPU_ALL_REGIONS, stream, n_regions=R)
    same = all(P.metrics_to_dict(x) == P.metrics_to_dict(y) for x, y in zip(got, want))
    step()
    P.talp_gpu_profile(ctx.ctx, True)
    P.talp_gpu_profile_read(ctx.ctx)
    l0 = P.talp_gpu_profile_read(ctx.ctx)["kernel_launches"]
    k = 10
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
    prof = P.talp_gpu_profile_read(ctx.ctx)
    P.talp_gpu_profile(ctx.ctx, False)
    sort_ms = prof["sort_ms"] / max(1, prof["sort_launches"])
    sweep_ms = prof["sweep_ms"] / max(1, prof["sweep_launches"])
    # the same records with TALP_GPU_GROUPED_BY_STREAM: the caller states the
    # grouping, each device's runs come from its stream ids, no first sweep
    bg, keep_g = P.batch_from_arrays(u.trace_id, u.devices_per_rank, u.region_window, arr["host_se"],
                                     arr["host_state"], u.host_off, arr["dev_se"], arr["dev_tag"], u.dev_off,
                                     P.TALP_GPU_GROUPED_BY_STREAM)

    def step_g():
        P.talp_gpu_ingest_events(ctx.ctx, [bg], stream)
        P.talp_gpu_region_metrics_device(ctx.ctx, [u.trace_id], P.TALP_GPU_ALL_REGIONS, out_dev.data_ptr(), stream)

    warm_until(step_g, 3, 0.5)
    got_g = P.talp_gpu_region_metrics(ctx.ctx, u.trace_id, P.TALP_GPU_ALL_REGIONS, stream, n_regions=R)
    same_g = all(P.metrics_to_dict(x) == P.metrics_to_dict(y) for x, y in zip(got_g, want))
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k):
        step_g()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_g = e0.elapsed_time(e1) / k
    ck = clocks.stop()
    n_dev = int(u.dev_off[-1])
    N = u.n_records
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_RECORD * n_dev / (sort_ms / 1000.0) / 1e9
    ctx.close()
    del arr, b, keep, bg, keep_g
    torch.cuda.empty_cache()
    return {
        "workload": "the plain large trace with each device's records grouped by stream (each stream in start "
                    "order), sorted by the library", "records_per_step": N, "steps": k, "ms_per_step": ms,
        "events_per_s": N / (ms / 1000.0),
        "sort_stage": {"ms": sort_ms, "device_records": n_dev, "first_sweep_ms": sweep_ms,
                       "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                    "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                                    "kernel": "sort stage (run finding, talp::fms_kernel and its plan and fix-up "
                                              "kernels), 17 B per device record"}},
        "bit_exact_vs_start_ordered": same,
        "grouped_by_stream_flag": {"ms_per_step": ms_g, "events_per_s": N / (ms_g / 1000.0),
                                   "bit_exact_vs_start_ordered": same_g,
                                   "form": "the same records ingested with TALP_GPU_GROUPED_BY_STREAM"},
        "gpu_launches": prof["kernel_launches"] - l0, "clocks": ck}


def default_extras(a, t=None, want=None):
    """Sub-objects of the default bench line: the served form and the plain
    form at the serving load (the p50/p99 query latency of the metric), the
    batched form against one trace per launch, and, on the plain trace `t`
    (results `want`), the sort stage, the concurrency profile and (at 25%)
    the raw activity-record adapter."""
    import copy
    sv = copy.copy(a)
    sv.warmup, sv.steps, sv.step_s, sv.sat_s, sv.plain_s, sv.native_s = 2, 10, 1.0, 0.0, 10.0, 5.0
    sv.jobs, sv.rate, sv.query_ms = 256, 2000.0, 10.0
    L = measure_serving(sv)
    pl = L["plain_same_load"]
    out = {
        "serving": {
            "workload": L["config"]["workload"], "seconds": sv.steps * sv.step_s, "warmup_s": sv.warmup * sv.step_s,
            "events_per_s": L["value"], "queries_per_s": L["served"]["queries_per_s"],
            "batches_per_s": L["served"]["batches_per_s"],
            "client_ms": L["latency_ms"], "native_client": L["native_client_latency_ms"],
            "library_ms": L["server_latency_ms"],
            "oracle_sampled_jobs": L["bit_exact_sampled_jobs"]["jobs"],
            "bit_exact_sampled_vs_oracle": L["bit_exact_sampled_jobs"]["exact"],
            "gpu_launches": L["gpu_launches"], "clocks": L["clocks"], "errors": L["errors"]},
        "serving_plain": {
            "workload": "the same jobs, arrivals and query period through the plain form: " + pl["form"],
            "seconds": sv.plain_s, "events_per_s": pl["events_per_s"], "queries_per_s": pl["queries_per_s"],
            "client_ms": {"p50": pl["p50_ms"], "p99": pl["p99_ms"]},
            "oracle_sampled_jobs": pl["bit_exact_sampled_jobs"]["jobs"],
            "bit_exact_sampled_vs_oracle": pl["bit_exact_sampled_jobs"]["exact"], "clocks": L["clocks_plain"]},
    }
    sp99, pp99 = L["latency_ms"]["p99"], pl["p99_ms"]
    out["serving"]["vs_plain"] = {"p99_plain_over_served": (pp99 / sp99) if sp99 and pp99 else None,
                                  "events_per_s_served_over_plain":
                                      L["value"] / pl["events_per_s"] if pl["events_per_s"] else None}
    bv = copy.copy(a)
    bv.traces, bv.ev_hi, bv.steps, bv.warmup = 4096, None, 10, 3
    B = measure_batched(bv)
    c = B["config"]
    out["batched"] = {
        "workload": c["workload"], "records_per_launch": c["records_per_step"], "ms_per_launch": B["ms_per_step"],
        "events_per_s": B["value"], "plain_one_trace_per_launch_events_per_s": c["plain_one_trace_per_launch_events_per_s"],
        "batched_over_plain": c["batched_over_plain"], "roofline_frac": B["roofline"]["frac"],
        "bit_exact_batched_vs_plain": c["bit_exact_batched_vs_plain"],
        "oracle_sampled_traces": c["oracle_sampled_traces"],
        "bit_exact_sampled_vs_oracle": c["bit_exact_sampled_vs_oracle"], "plan": c["plan"],
        "gpu_launches": B["gpu_launches"], "clocks": B["clocks"]}
    ok = (out["serving"]["bit_exact_sampled_vs_oracle"] and out["serving_plain"]["bit_exact_sampled_vs_oracle"]
          and not out["serving"]["errors"] and out["batched"]["bit_exact_sampled_vs_oracle"]
          and out["batched"]["bit_exact_batched_vs_plain"])
    if t is not None:
        out["sort_stage"] = measure_sort_stage(a, t, want)
        cv = copy.copy(a)
        cv.steps, cv.warmup, cv.scale = 5, 3, 1.0
        C = measure_concurrency(cv, t)
        out["concurrency"] = {
            "workload": C["config"]["workload"], "records_per_call": C["config"]["records_per_step"],
            "ms_per_call": C["ms_per_step"], "records_per_s": C["value"], "roofline_frac": C["roofline"]["frac"],
            "bit_exact_rank0_vs_oracle": C["config"]["bit_exact_rank0_vs_oracle"],
            "gpu_launches": C["gpu_launches"], "clocks": C["clocks"]}
        rv = copy.copy(a)
        rv.steps, rv.warmup, rv.scale, rv.hold_calls = 10, 3, 0.25, 1
        W = measure_raw(rv)
        out["raw"] = {
            "workload": W["config"]["workload"], "records_per_step": W["config"]["records_per_step"],
            "ms_per_step": W["ms_per_step"], "events_per_s": W["value"],
            "lanes_in_start_order_ms_per_step": W["config"]["lanes_in_start_order_ms_per_step"],
            "roofline_frac": W["roofline"]["frac"], "bit_exact_raw_vs_lanes": W["config"]["bit_exact_raw_vs_lanes"],
            "gpu_launches": W["gpu_launches"], "clocks": W["clocks"]}
        ok = (ok and out["sort_stage"]["bit_exact_vs_start_ordered"]
              and out["sort_stage"]["grouped_by_stream_flag"]["bit_exact_vs_start_ordered"]
              and out["concurrency"]["bit_exact_rank0_vs_oracle"] and out["raw"]["bit_exact_raw_vs_lanes"])
    out["_rc"] = 0 if ok else 1
    return out


if __name__ == "__main__":
    sys.exit(main())
