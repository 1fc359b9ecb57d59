/*
 * talp_gpu.h -- C ABI of the B300 efficiency-metric reducer.
 *
 * The library turns per-rank host-state intervals and per-device activity
 * records into the extended POP efficiency hierarchy of "Hardware-Agnostic
 * and Insightful Efficiency Metrics for Accelerated Systems" (arXiv
 * 2603.26576), per monitoring region:
 *   host tree   (Sec. 4.1, Eqs. 6-8): Host Hybrid Parallel Efficiency =
 *               MPI Parallel Efficiency (= load balance x communication
 *               efficiency, offloading counted as useful) x Device Offload
 *               Efficiency;
 *   device tree (Sec. 4.1, Eqs. 9-12): Device Parallel Efficiency = load
 *               balance x communication efficiency x orchestration efficiency,
 *               over the kernel / memory-operation / idle occupancy of every
 *               device obtained by the flattening of Sec. 4.2.
 * All interval arithmetic is exact int64 nanoseconds on the GPU; the nine
 * ratios are formed in FP64 with a fixed expression order.
 * Beyond the two trees: raw activity buffers in completion order
 * (talp_gpu_ingest_raw), the per-device concurrency profile, POP scaling
 * factors across runs, and a host tree with threads (a variant the paper
 * does not define, equal to the host tree with one thread per process).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Intervals are half open [start, end) in int64 ns; end == start adds 0;
 *    end < start is invalid input.
 *  - A record is 16 bytes {int64 start, int64 end} in an array `*_se`
 *    (row j at se[2j], se[2j+1]) plus one byte in a parallel array:
 *      host:   state, one of TALP_HOST_* (Sec. 4.1 host states);
 *      device: tag = kind << 5 | stream, kind one of TALP_DEV_* (kernel or a
 *              memory operation, Sec. 4.1 / 4.2), stream 0..31.
 *  - Records are grouped by CSR offsets: host records by rank
 *    (host_off[n_ranks + 1]); device records by device, devices numbered
 *    rank-major (rank 0's devices first), dev_off[m + 1] with
 *    m = sum(devices_per_rank).  A device owns no records of other ranks.
 *  - A region is one window [begin, end) per rank; every host interval of a
 *    rank and every record of its devices is clipped to it (regions are
 *    independent; nesting is allowed).
 *  - A ratio whose denominator is 0 reads 1 (no loss attributable to that
 *    factor); E == 0 sets TALP_GPU_M_EMPTY and every ratio to 1.
 *  - Errors are returned as talp_gpu_status; nothing throws across the ABI.
 *    talp_gpu_last_error() gives a message for the calling thread.
 *  - `stream` is a cudaStream_t (0 = legacy default stream).  Calls that
 *    return results to the host synchronise that stream; the others are
 *    stream ordered and return once the work is enqueued.
 *  - Every call is safe from one host thread per context; a context must
 *    not be used by two threads at once.
 */
#ifndef TALP_GPU_H
#define TALP_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TALP_GPU_ABI_VERSION 1
#define TALP_GPU_MAX_REGIONS 8
#define TALP_GPU_ALL ((uint64_t)-1)             /* talp_gpu_reset: every trace */
#define TALP_GPU_ALL_REGIONS ((uint32_t)-1)     /* region selector: all regions */

typedef struct talp_gpu_ctx talp_gpu_ctx;       /* opaque; owns all device state */

typedef enum {
    TALP_GPU_OK = 0,
    TALP_GPU_EINVAL = -1,      /* bad argument or invalid record detected */
    TALP_GPU_ENOMEM = -2,      /* HBM budget or device allocation exhausted */
    TALP_GPU_ECUDA = -3,       /* a CUDA runtime call failed */
    TALP_GPU_ETIMEDOUT = -4,   /* a bounded device-side wait ran out */
    TALP_GPU_ENOTFOUND = -5,   /* unknown trace id or job id */
    TALP_GPU_EBUSY = -6        /* resource in use (serving slot, pending work) */
} talp_gpu_status;

/* host states (Sec. 4.1): useful, device offloading, MPI calls */
enum { TALP_HOST_USEFUL = 0, TALP_HOST_OFFLOAD = 1, TALP_HOST_MPI = 2 };
/* device record kinds: kernel = useful; the rest are memory operations
 * (GPU-GPU and CPU-GPU transfers and memsets, Sec. 4.1 / 4.2) */
enum { TALP_DEV_KERNEL = 0, TALP_DEV_H2D = 1, TALP_DEV_D2H = 2, TALP_DEV_D2D = 3, TALP_DEV_MEMSET = 4 };
#define TALP_DEV_TAG(kind, stream) ((uint8_t)((((unsigned)(kind)) << 5) | (((unsigned)(stream)) & 31u)))

/* talp_gpu_trace_batch.flags */
#define TALP_GPU_DEVICE_PTRS     0x1u  /* host_se/host_state/dev_se/dev_tag are device pointers */
#define TALP_GPU_SORTED_BY_START 0x2u  /* caller asserts each device's records are in start order */
#define TALP_GPU_APPEND          0x4u  /* fold into the trace's running state (later time slice) */
#define TALP_GPU_NOT_SORTED      0x10u /* caller hint: device records are out of start order (e.g.
                                        * grouped by stream): every device goes straight to the
                                        * sort stage without a first sweep; one found in order is
                                        * swept from its own records.  Not with SORTED_BY_START. */
#define TALP_GPU_GROUPED_BY_STREAM 0x20u /* caller asserts that, on every device, each stretch of
                                        * consecutive records on one stream is in start order (the
                                        * order per-stream activity buffers deliver when handed over
                                        * one stream after another, Sec. 4.2): the stretches are the
                                        * device's sorted runs, found from the stream ids of its tags,
                                        * and the device goes straight to the sort stage.  A stretch
                                        * out of start order makes the next result call return
                                        * TALP_GPU_EINVAL.  A device of one stretch, or of more than
                                        * 16, is handled as under NOT_SORTED.  Not with
                                        * SORTED_BY_START or NOT_SORTED. */

/*
 * One trace (or one later time slice of it with TALP_GPU_APPEND).
 *
 * Pointers marked "host" are always host memory and are read during the
 * call.  The four record arrays are host memory, or device memory of the
 * context's GPU when TALP_GPU_DEVICE_PTRS is set; device record arrays must
 * start on a 16-byte boundary and stay valid and unmodified until `stream`
 * has passed the ingest call.  Host record arrays are copied during the call
 * (pinned memory makes the copy faster; pageable memory works).
 *
 * Without TALP_GPU_SORTED_BY_START the library checks the order of every
 * device's records on the GPU and sorts the devices that need it.  With the
 * flag, a device found out of order makes the next result call return
 * TALP_GPU_EINVAL.
 *
 * TALP_GPU_APPEND continues an existing trace: the shape (n_ranks,
 * devices_per_rank, n_regions) must match, every device's new records must
 * start no earlier than its last ingested record, and the windows given here
 * replace the stored ones.  Without APPEND an existing trace of the same id is
 * replaced.
 */
typedef struct {
    uint64_t trace_id;
    uint32_t n_ranks;                  /* n >= 1 */
    uint32_t n_regions;                /* 1 .. TALP_GPU_MAX_REGIONS */
    uint32_t flags;
    uint32_t reserved;                 /* must be 0 */
    const uint32_t *devices_per_rank;  /* host [n_ranks] */
    const int64_t *region_window;      /* host [n_regions][n_ranks][2] = [begin, end) */
    const int64_t *host_se;            /* [N_host][2] */
    const uint8_t *host_state;         /* [N_host] */
    const uint64_t *host_off;          /* host [n_ranks + 1], host_off[0] == 0 */
    const int64_t *dev_se;             /* [N_dev][2] */
    const uint8_t *dev_tag;            /* [N_dev] */
    const uint64_t *dev_off;           /* host [m + 1], dev_off[0] == 0 */
} talp_gpu_trace_batch;

/* talp_gpu_metrics.flags */
#define TALP_GPU_M_EMPTY          0x1u  /* E == 0: every ratio reported as 1 */
#define TALP_GPU_M_HOST_NOT_TILED 0x2u  /* some rank's host intervals do not sum to its window */
#define TALP_GPU_M_NO_DEVICES     0x4u  /* m == 0: device ratios reported as 1 */
#define TALP_GPU_M_INVALID        0x100u /* invalid record seen (end < start, bad kind/state) */
#define TALP_GPU_M_UNSORTED       0x200u /* out-of-order device records under SORTED_BY_START/APPEND */
#define TALP_GPU_M_TIMEOUT        0x400u /* a bounded device-side wait ran out while ingesting */

/*
 * Metrics of one region of one trace.  Sums are over ranks (host) or devices
 * (device) of the region-clipped times; every time is int64 ns.
 */
typedef struct {
    uint64_t trace_id;
    uint32_t region;
    uint32_t flags;                    /* TALP_GPU_M_* */
    uint32_t n_ranks;                  /* n */
    uint32_t m_devices;                /* m */
    int64_t elapsed_ns;                /* E = max_i (U_i + W_i + MPI_i), Eq. 1 */
    int64_t sum_useful;                /* sum_i U_i (Eq. 2) */
    int64_t sum_offload;               /* sum_i W_i */
    int64_t sum_mpi;                   /* sum_i MPI_i */
    int64_t max_useful_offload;        /* max_i (U_i + W_i) */
    int64_t sum_kernel;                /* sum_g D_K,g  (kernel union per device) */
    int64_t max_kernel;                /* max_g D_K,g */
    int64_t max_busy;                  /* max_g (D_K,g + D_M,g) */
    int64_t sum_mem;                   /* sum_g D_M,g  (transfers not under kernels) */
    int64_t sum_idle;                  /* sum_g (window_g - D_K,g - D_M,g) */
    int64_t sum_hidden_mem;            /* sum_g |transfers under kernels| */
    double host_pe;                    /* Eq. 6  sum U / (E n) */
    double host_mpi_pe;                /* Eq. 7  sum (U+W) / (E n) */
    double host_mpi_lb;                /* sum (U+W) / (n max (U+W)) */
    double host_mpi_ce;                /* max (U+W) / E */
    double host_oe;                    /* Eq. 8  sum U / sum (U+W) */
    double dev_pe;                     /* Eq. 9  sum D_K / (E m) */
    double dev_lb;                     /* Eq. 10 sum D_K / (m max D_K) */
    double dev_ce;                     /* Eq. 11 max D_K / max (D_K + D_M) */
    double dev_oe;                     /* Eq. 12 max (D_K + D_M) / E */
} talp_gpu_metrics;

/* ---------------------------------------------------------------- context */

/*
 * Create a context on CUDA device `device`.  (Library service, no passage:
 * the context holds the per-trace running state that the at-runtime queries
 * of Sec. 3.2 read.)  hbm_budget_bytes caps the device memory the context
 * may hold (traces, staging, workspace); 0 means 90% of the device's free
 * memory at creation.  *out receives the context; the caller owns it and
 * frees it with talp_gpu_destroy.
 * Errors: EINVAL (null out, bad device), ECUDA.
 */
talp_gpu_status talp_gpu_create(talp_gpu_ctx **out, int device, size_t hbm_budget_bytes);

/* Free every device buffer and the context.  (Library service, no passage.)
 * NULL is accepted.  Synchronises the context's device work first.
 * Errors: EBUSY (nothing freed) while a plan or a server created on the
 * context still exists: destroy those first. */
talp_gpu_status talp_gpu_destroy(talp_gpu_ctx *ctx);

/* ------------------------------------------------------------------ ingest */

/*
 * Ingest n_batches traces (the plain form is n_batches == 1; larger n is the
 * batched form: every trace is reduced by the same persistent launch
 * sequence).  Validation of the headers happens on the host before anything
 * is enqueued (EINVAL, nothing changed); validation of the records happens on
 * the GPU and surfaces as EINVAL from the next result call for that trace.
 * Admission: ENOMEM is returned before any allocation when the traces would
 * exceed the context's HBM budget.  The call is stream ordered.
 * The trace's per-rank and per-device partial sums stay on the device
 * (Sec. 4.2 flattening and the host-state sums of Sec. 4.1).
 */
talp_gpu_status talp_gpu_ingest_events(talp_gpu_ctx *ctx, const talp_gpu_trace_batch *batches,
                                       size_t n_batches, void *stream);

/*
 * Raw activity records (Sec. 4.2: device records reach the tool in buffers,
 * delivered when full or flushed, with the records of all of a process's
 * devices and streams interleaved in completion order).  Same as
 * talp_gpu_trace_batch except for the device records: rank i's records are
 * raw_se / raw_tag / raw_dev [raw_off[i] .. raw_off[i+1]), in delivery
 * order, raw_dev being the record's device within its rank (0 ..
 * devices_per_rank[i] - 1, at most 8 devices per rank).  Records of one
 * stream must be delivered in start order (a stream executes in order); the
 * streams may interleave arbitrarily.  (A stream found out of start order
 * makes the next result call for the trace return EINVAL.)
 *
 * TALP_GPU_HOLD_BACK streams a trace's buffers over several calls.  A later
 * buffer may still bring a record that starts before records of other
 * streams already delivered, so, per device, only the records starting at
 * or before its watermark W = min over the device's declared streams of
 * their last delivered start are folded; the others are held back on the
 * GPU and delivered again, ahead of the next call's records of the trace.
 * stream_mask[i * 8 + d] declares the streams (bit s = stream s) of device
 * d of rank i; a declared stream that has delivered nothing yet holds its
 * device's watermark below every record.  A call for the trace without
 * TALP_GPU_HOLD_BACK folds every held record (a flush) and ends the hold
 * state; so do a call without TALP_GPU_APPEND and talp_gpu_reset.  The
 * first hold-back call of a trace may come without APPEND (it creates the
 * trace), later ones take APPEND.
 */
#define TALP_GPU_HOLD_BACK 0x8u   /* raw batches: hold back records a later buffer may precede */

typedef struct {
    uint64_t trace_id;
    uint32_t n_ranks;
    uint32_t n_regions;
    uint32_t flags;                    /* TALP_GPU_DEVICE_PTRS (all record arrays), TALP_GPU_APPEND,
                                          TALP_GPU_HOLD_BACK */
    uint32_t reserved;                 /* must be 0 */
    const uint32_t *devices_per_rank;  /* host [n_ranks], each <= 8 */
    const int64_t *region_window;      /* host [n_regions][n_ranks][2] */
    const int64_t *host_se;            /* [N_host][2] */
    const uint8_t *host_state;         /* [N_host] */
    const uint64_t *host_off;          /* host [n_ranks + 1] */
    const int64_t *raw_se;             /* [N_raw][2] */
    const uint8_t *raw_tag;            /* [N_raw] kind << 5 | stream */
    const uint8_t *raw_dev;            /* [N_raw] device within the rank */
    const uint64_t *raw_off;           /* host [n_ranks + 1], raw_off[0] == 0 */
    const uint32_t *stream_mask;       /* host [n_ranks][8] declared streams; needed with HOLD_BACK, else
                                          may be NULL */
} talp_gpu_raw_batch;

/*
 * Ingest raw activity records: a stable scatter on the GPU groups every
 * rank's records by (device, stream) into per-device lanes, each stream in
 * delivery (= start) order, then (TALP_GPU_HOLD_BACK) splits each lane at
 * its device's watermark, and the lanes go through talp_gpu_ingest_events
 * without TALP_GPU_SORTED_BY_START (the out-of-order devices are merged by
 * start on the GPU).  Synchronises `stream` once, to read each device's
 * record count.  A trace appears at most once per call.  Errors: those of
 * talp_gpu_ingest_events; EINVAL for a record naming a device its rank does
 * not have, more than 8 devices in a rank, HOLD_BACK without stream masks,
 * a shape that differs from the held records' trace, 2^32 records in one
 * rank of a hold-back call, and a record on a stream its device does not
 * declare (found on the GPU; the trace's held records are then dropped).
 */
talp_gpu_status talp_gpu_ingest_raw(talp_gpu_ctx *ctx, const talp_gpu_raw_batch *batches, size_t n_batches,
                                    void *stream);

/*
 * Number of raw records of trace `trace_id` held back by TALP_GPU_HOLD_BACK
 * calls and not folded yet (0 for a trace without hold state).  Host call,
 * no GPU work.  Errors: EINVAL (null argument).
 */
talp_gpu_status talp_gpu_raw_held(talp_gpu_ctx *ctx, uint64_t trace_id, uint64_t *out_host);

/* ----------------------------------------------------------------- results */

/*
 * Metrics of `region` (or every region with TALP_GPU_ALL_REGIONS, written to
 * out_host[0 .. n_regions-1]) of trace `trace_id`: the Eqs. 1 and 6-12 ratios
 * formed on the GPU from its sums.  Synchronises `stream`.
 * Errors: ENOTFOUND (unknown trace), EINVAL (bad region, or invalid records
 * were ingested: out_host is still written and its flags say why),
 * ETIMEDOUT (a device-side bounded wait ran out during ingest), ECUDA.
 */
talp_gpu_status talp_gpu_region_metrics(talp_gpu_ctx *ctx, uint64_t trace_id, uint32_t region,
                                        talp_gpu_metrics *out_host, void *stream);

/*
 * Metrics of one region for n traces with one launch and one copy:
 * out_host[k] belongs to trace_ids[k] (the same Eqs. 1 and 6-12 per trace;
 * batching serves many at-runtime queries at once, Sec. 3.2).  trace_ids
 * and out_host are host memory [n].  Same errors as above (the first
 * failing trace decides the status; every entry is written).
 */
talp_gpu_status talp_gpu_region_metrics_batch(talp_gpu_ctx *ctx, const uint64_t *trace_ids, size_t n,
                                              uint32_t region, talp_gpu_metrics *out_host, void *stream);

/*
 * Stream-ordered variant: writes the n metrics structs to device memory
 * out_device (n entries, 8-byte aligned) without synchronising.  Record
 * problems are reported only through the flags of the written structs.
 */
talp_gpu_status talp_gpu_region_metrics_device(talp_gpu_ctx *ctx, const uint64_t *trace_ids, size_t n,
                                               uint32_t region, talp_gpu_metrics *out_device,
                                               void *stream);

/*
 * Sharded reduction (one trace split over several GPUs or contexts by whole
 * ranks, each rank with all of its devices): parts[0 .. n_parts-1] are the
 * talp_gpu_metrics of one region computed on each shard (host memory, same
 * trace_id and region).  Their integer aggregates combine exactly -- E
 * (Eq. 1, a maximum over ranks) and the maxima of Eqs. 7-12 by max, the
 * sums and the rank/device counts by addition, the status flags by or --
 * and one kernel forms the nine ratios from the combined aggregates, so
 * out_host equals the metrics of the whole trace bit for bit.  The shards'
 * own ratios are ignored.  Synchronises `stream`.
 * Errors: EINVAL (no parts, more than 2^20, mixed traces or regions, or a
 * part carrying the flag of invalid records), ETIMEDOUT, ECUDA.
 */
talp_gpu_status talp_gpu_metrics_combine(talp_gpu_ctx *ctx, const talp_gpu_metrics *parts, size_t n_parts,
                                         talp_gpu_metrics *out_host, void *stream);

/*
 * Host tree with threads (a variant: the paper's host tree, Sec. 4.1
 * Eqs. 6-8, has one set of host intervals per MPI rank and no thread level).
 * Ingest the trace with one host unit per thread -- n_ranks = the number of
 * threads nT, each thread's useful / offload / MPI intervals as its unit's
 * host records, each thread with its process's windows, the devices on any
 * unit (normally the master thread's) -- and group the units into processes
 * with proc_off (host memory, n_procs + 1 entries): process i owns units
 * proc_off[i] .. proc_off[i+1]-1, T_i >= 1 of them.  With B = U + W per
 * thread and M_i = the largest B of process i (its busiest thread):
 *   E         = max over threads (U + W + MPI)            (Eq. 1 over threads)
 *   pe        = sum U / (E nT)                            (Eq. 6 over threads)
 *   mpi_pe    = sum_i T_i M_i / (E nT)  = mpi_lb x mpi_ce (Eq. 7, the busiest
 *     mpi_lb  = sum_i T_i M_i / (nT max_i M_i)             thread standing for
 *     mpi_ce  = max_i M_i / E                              its process)
 *   thread_lb = sum B / sum_i T_i M_i                     (Eq. 10's form inside
 *                                                          each process)
 *   oe        = sum U / sum B                             (Eq. 8 over threads)
 * so pe = mpi_pe x thread_lb x oe, and with one thread per process every
 * value equals talp_gpu_region_metrics' host tree bit for bit.  E is the
 * same as talp_gpu_region_metrics' (threads as units), so its device tree
 * holds unchanged.  FP64 on the GPU in the order written; 0/0 reads 1; E = 0
 * sets TALP_GPU_M_EMPTY with every ratio 1.  Sums are int64: nT x E must
 * stay below 2^63.
 * out_host[0] (or out_host[0 .. n_regions-1] with TALP_GPU_ALL_REGIONS),
 * host memory; synchronises `stream`.
 * Errors: ENOTFOUND (unknown trace), EINVAL (bad region; proc_off not
 * starting at 0, not strictly increasing, or not ending at the trace's
 * n_ranks; invalid records ingested: out_host is still written and its
 * flags say why), ETIMEDOUT, ECUDA.
 */
typedef struct {
    uint64_t trace_id;
    uint32_t region;
    uint32_t flags;                    /* TALP_GPU_M_EMPTY and the status flags */
    uint32_t n_procs, n_threads;
    int64_t elapsed_ns;                /* E = max over threads (U + W + MPI) */
    int64_t sum_useful;                /* sum over threads U */
    int64_t sum_offload;               /* sum over threads W */
    int64_t sum_busiest;               /* sum_i T_i M_i */
    int64_t max_busiest;               /* max_i M_i */
    double pe, mpi_pe, mpi_lb, mpi_ce, thread_lb, oe;
} talp_gpu_thread_tree;
talp_gpu_status talp_gpu_thread_metrics(talp_gpu_ctx *ctx, uint64_t trace_id, uint32_t region,
                                        const uint32_t *proc_off, uint32_t n_procs,
                                        talp_gpu_thread_tree *out_host, void *stream);
/*
 * Stream-ordered variant: writes the records to device memory out_device (one
 * per region, 8-byte aligned) without synchronising; proc_off is still host
 * memory, read during the call.  Record problems are reported only through
 * the flags of the written records.
 */
talp_gpu_status talp_gpu_thread_metrics_device(talp_gpu_ctx *ctx, uint64_t trace_id, uint32_t region,
                                               const uint32_t *proc_off, uint32_t n_procs,
                                               talp_gpu_thread_tree *out_device, void *stream);
/*
 * Sharded thread tree (one trace split over GPUs or contexts by whole
 * processes, each with all of its threads and their devices): parts are the
 * records of one region computed on each shard (host memory, same trace_id
 * and region).  E and max_busiest combine by max, the sums and the process
 * and thread counts by addition, the status flags by or, and one kernel
 * forms the six ratios from them, so the result equals the whole trace's
 * bit for bit.  out_host: one record; synchronises `stream`.
 * Errors: EINVAL (no parts, more than 2^20, mixed traces or regions, a part
 * carrying the flag of invalid records), ETIMEDOUT, ECUDA.
 */
talp_gpu_status talp_gpu_thread_metrics_combine(talp_gpu_ctx *ctx, const talp_gpu_thread_tree *parts,
                                                size_t n_parts, talp_gpu_thread_tree *out_host, void *stream);

/*
 * Scalability across runs: POP's second branch, which needs several runs
 * and which TALP leaves to the user (Sec. 3.3).  runs[0 .. n_runs-1] are
 * the metrics of one region (the same region index) of runs of one
 * application at different scales, runs[ref] the reference.  For run r:
 *   speedup         = E_ref / E_r
 *   host_comp_scal  strong: sumU_ref / sumU_r
 *                   weak:   (sumU_ref * n_r) / (sumU_r * n_ref)
 *   host_global_eff = PE_host_r * host_comp_scal
 *   dev_comp_scal   the same with the kernel sums and m
 *   dev_global_eff  = PE_dev_r * dev_comp_scal
 * FP64 on the GPU, round to nearest in the order written; a zero
 * denominator reads 1.  out_host[n_runs], host memory; synchronises stream.
 * The hardware-counter children of computation scalability (IPC,
 * instructions, frequency) are not covered.
 * Errors: EINVAL (no runs, ref out of range, bad mode, mixed regions), ECUDA.
 */
#define TALP_GPU_SCALING_STRONG 0u
#define TALP_GPU_SCALING_WEAK 1u
typedef struct {
    uint64_t trace_id;
    uint32_t region;
    uint32_t flags;                    /* the run's TALP_GPU_M_* flags */
    uint32_t n_ranks, m_devices;
    double speedup;
    double host_comp_scal, host_global_eff;
    double dev_comp_scal, dev_global_eff;
} talp_gpu_scaling;
talp_gpu_status talp_gpu_scalability(talp_gpu_ctx *ctx, const talp_gpu_metrics *runs, size_t n_runs, size_t ref,
                                     uint32_t mode, talp_gpu_scaling *out_host, void *stream);

/*
 * Raw per-unit times of one region (TALP also reports raw times so users can
 * form their own indicators): host_out [n_ranks][3] = useful, offload, MPI
 * per rank; dev_out [m][3] = kernel union D_K, memory-operation union, busy
 * union B per device (D_M = B - D_K).  Either pointer may be NULL.  Host
 * memory; synchronises `stream`.
 */
talp_gpu_status talp_gpu_unit_sums(talp_gpu_ctx *ctx, uint64_t trace_id, uint32_t region,
                                   int64_t *host_out, int64_t *dev_out, void *stream);

/*
 * Concurrency profile of every device of one trace in one region: the
 * per-stream occupancy the paper leaves to future work (Sec. 4.1, device
 * states; the streams are merged here).  With a device's records clipped to
 * its rank's window and c(t) the number of them active at time t,
 *   out_host[g][0][k-1] = |{t : c(t) >= k}|            k = 1 .. TALP_GPU_CONC_LEVELS,
 *   out_host[g][1][k-1] = the same over kernel records,
 * int64 ns, host memory [m][2][TALP_GPU_CONC_LEVELS].  Level 1 equals the
 * busy union (resp. the kernel union) of the flattening (Sec. 4.2).
 * `b` is read as for talp_gpu_ingest_events (host records are ignored, the
 * device records must be in start order per device; TALP_GPU_APPEND is not
 * used); nothing is stored.  Synchronises `stream`.
 * Errors: EINVAL (bad header or region; a record with end < start or a bad
 * kind; device records out of start order: out_host is still written),
 * ENOMEM, ECUDA.
 */
#define TALP_GPU_CONC_LEVELS 8
talp_gpu_status talp_gpu_concurrency(talp_gpu_ctx *ctx, const talp_gpu_trace_batch *b, uint32_t region,
                                     int64_t *out_host, void *stream);

/* ------------------------------------------------------------ batched plans */

/*
 * A plan is the batched form: the whole reduction of many traces (of uneven
 * rank, device and record counts) -- prep, sweep, fix-up, the sort stage when
 * records may be out of order, and the finalize of every region of every
 * trace -- recorded once as a CUDA graph and replayed by talp_gpu_plan_launch
 * as one graph launch; its segment tables are uploaded once, when the plan
 * is created.  Each trace's
 * sums are the same as after talp_gpu_ingest_events of that trace alone
 * (Sec. 4.1, 4.2, Eqs. 1-12 per trace and region); the traces also stay in
 * the context (talp_gpu_region_metrics etc. work on them after a launch).
 *
 * batches:    n traces; every one with TALP_GPU_DEVICE_PTRS and without
 *             TALP_GPU_APPEND.  The record arrays must stay at the same
 *             device addresses for the plan's lifetime; their contents may
 *             change between launches (shapes and offsets may not).
 * plan_flags: TALP_GPU_PLAN_AUTOTUNE times every sweep shape (records per
 *             lane, warps, pipeline stages) x per-segment cost x work split
 *             (one fixed slice of the records per warp, or 16 slices per
 *             warp handed to the warps as they come free) on these traces
 *             and keeps the fastest; the choice is also remembered by the
 *             context for later ingests of the same size class.
 * Errors: EINVAL, ENOMEM (admission: plan workspace + new traces), EBUSY
 * (a trace id in use by a plan with another shape), ECUDA.
 * A trace used by a plan cannot be reset or re-shaped (EBUSY) until the plan
 * is destroyed.
 */
#define TALP_GPU_PLAN_AUTOTUNE 0x1u

typedef struct talp_gpu_plan talp_gpu_plan;

typedef struct {
    uint64_t n_metrics;                /* sum of n_regions over the plan's traces */
    uint64_t records;                  /* records reduced per launch */
    uint64_t segments;                 /* device + host segments */
    uint32_t kernels_per_launch;       /* kernels in the graph */
    uint32_t sweep_items;              /* chosen sweep shape: records per lane per tile */
    uint32_t sweep_warps;              /*   warps per CTA */
    uint32_t sweep_stages;             /*   TMA pipeline stages per warp */
    uint32_t tiles_per_warp;           /*   minimum tiles per warp (grid sizing) */
    uint32_t sweep_grid;               /*   CTAs of the sweep launch */
    uint32_t slices_per_warp;          /*   0: one fixed slice of the records per warp; k: k slices per
                                        *   warp handed to the warps as they come free */
} talp_gpu_plan_stats;

talp_gpu_status talp_gpu_plan_create(talp_gpu_ctx *ctx, const talp_gpu_trace_batch *batches, size_t n,
                                     uint32_t plan_flags, talp_gpu_plan **out);
/* Enqueue one replay of the plan's graph on `stream` (stream ordered). */
talp_gpu_status talp_gpu_plan_launch(talp_gpu_plan *plan, void *stream);
/* Copy the metrics of the last launch to out_host[n_metrics] (traces in plan
 * order, regions 0..R-1 each) and synchronise `stream`; EINVAL/ETIMEDOUT
 * as for talp_gpu_region_metrics (out_host is written either way). */
talp_gpu_status talp_gpu_plan_metrics(talp_gpu_plan *plan, talp_gpu_metrics *out_host, void *stream);
talp_gpu_status talp_gpu_plan_info(talp_gpu_plan *plan, talp_gpu_plan_stats *out);
/* Synchronise the device and free the plan (the traces stay). NULL is accepted. */
talp_gpu_status talp_gpu_plan_destroy(talp_gpu_plan *plan);

/* ----------------------------------------------------------------- serving */

/*
 * The served form: at-runtime monitoring of many jobs (TALP answers queries
 * while the application runs, Sec. 3.2).  Each job is a trace whose
 * per-rank/per-device running state (sums and carries of Sec. 4.1/4.2)
 * stays on the device.  Client threads submit the job's records as time
 * slices (talp_gpu_server_submit) and ask for metrics (talp_gpu_server_query)
 * concurrently.  A server thread batches continuously: every job's pending
 * slice joins the next fold wave (one APPEND ingest of all of them), waves
 * are enqueued back to back while earlier ones run, and pending queries are
 * batched into one finalize launch on a separate stream, ordered after the
 * wave that holds their data.  A query returns the metrics of the job with
 * at least every slice submitted before it folded in; the result does not
 * depend on what else is in flight.
 *
 * Admission: talp_gpu_server_open_job fails with EBUSY when all job slots
 * are taken and with ENOMEM when the job's state would exceed the context's
 * HBM budget; closing a job frees its slot and memory.
 *
 * Slices: host memory, copied during the call; flags may only hold
 * TALP_GPU_SORTED_BY_START (APPEND is implied after the first slice); a
 * job's slices must come in time order per device (a slice may be out of
 * order inside itself: it is sorted on the device).  Records per slice are
 * limited by max_slice_records.
 */
typedef struct talp_gpu_server talp_gpu_server;

typedef struct {
    uint32_t max_jobs;                 /* job slots (admission) */
    uint32_t max_slice_records;        /* host + device records per submitted slice */
    uint32_t staging_slices;           /* pinned staging buffers (slices in flight) */
    uint32_t reserved;
} talp_gpu_server_config;

typedef struct {
    uint64_t slices_submitted, slices_folded;
    uint64_t records_folded;
    uint64_t waves;                    /* fold waves launched */
    uint64_t queries, query_batches;   /* answered queries, finalize launches for them */
    double query_p50_ms, query_p99_ms, query_max_ms;   /* submit-to-answer latency of queries */
    uint32_t jobs_open, reserved;
} talp_gpu_server_stats;

talp_gpu_status talp_gpu_server_create(talp_gpu_ctx *ctx, const talp_gpu_server_config *cfg,
                                       talp_gpu_server **out);
/* Admit a job: n_ranks, devices_per_rank[n_ranks], n_regions and the region
 * windows [n_regions][n_ranks][2] as in talp_gpu_trace_batch. */
talp_gpu_status talp_gpu_server_open_job(talp_gpu_server *srv, uint64_t job_id, uint32_t n_ranks,
                                         const uint32_t *devices_per_rank, uint32_t n_regions,
                                         const int64_t *region_window);
/* Queue one time slice of a job (the batch's trace_id, n_ranks, n_regions,
 * devices_per_rank and region_window are ignored: the job's are used). */
talp_gpu_status talp_gpu_server_submit(talp_gpu_server *srv, uint64_t job_id, const talp_gpu_trace_batch *slice);
/* Queue one raw activity buffer of a job (talp_gpu_raw_batch; its
 * trace_id, n_ranks, n_regions, devices_per_rank and region_window are
 * ignored: the job's are used; at most 8 devices per rank).  Flags:
 * TALP_GPU_HOLD_BACK only.  With it, the wave folds the records up to each
 * device's watermark and holds the rest back on the GPU (stream_mask, [n][8],
 * declares the streams); without it, the buffer and
 * every held record of the job are folded.  A query answers over the folded
 * records.  The job's declared streams are the union of all masks it was
 * given.  The buffer is checked during the call: EINVAL for a record naming
 * a device its rank does not have or (with HOLD_BACK) a stream its device
 * does not declare, and nothing is queued.  Records per buffer are limited
 * by max_slice_records; the record arrays are host memory, copied during
 * the call. */
talp_gpu_status talp_gpu_server_submit_raw(talp_gpu_server *srv, uint64_t job_id, const talp_gpu_raw_batch *buf);
/* Metrics of one region (or TALP_GPU_ALL_REGIONS: out_host[n_regions]);
 * blocks until answered.  EINVAL when the job's records were invalid. */
talp_gpu_status talp_gpu_server_query(talp_gpu_server *srv, uint64_t job_id, uint32_t region,
                                      talp_gpu_metrics *out_host);
/* Host tree with threads of one region (or TALP_GPU_ALL_REGIONS:
 * out_host[n_regions]) over the same state as talp_gpu_server_query: the
 * job's host units are threads, grouped into processes by proc_off (host
 * memory, n_procs + 1 entries, read while the call waits; the rules of
 * talp_gpu_thread_metrics).  Batched with the other queries on the query
 * stream; blocks until answered.  EINVAL for a bad process table or when
 * the job's records were invalid; ENOMEM when no room for the table. */
talp_gpu_status talp_gpu_server_query_threads(talp_gpu_server *srv, uint64_t job_id, uint32_t region,
                                              const uint32_t *proc_off, uint32_t n_procs,
                                              talp_gpu_thread_tree *out_host);
/* Wait until everything submitted so far is folded. */
talp_gpu_status talp_gpu_server_drain(talp_gpu_server *srv);
talp_gpu_status talp_gpu_server_close_job(talp_gpu_server *srv, uint64_t job_id);
talp_gpu_status talp_gpu_server_info(talp_gpu_server *srv, talp_gpu_server_stats *out);
/* Stop the server threads, close every job, free the server. NULL is accepted. */
talp_gpu_status talp_gpu_server_destroy(talp_gpu_server *srv);

/* Drop trace_id's state and return its HBM (TALP_GPU_ALL: every trace).
 * This ends a monitored run's running state: TALP keeps accumulating
 * region times until the run ends and queries read them meanwhile
 * (Sec. 3.2); a new trace of the same id starts from zero.  Synchronises
 * the context's work on the trace first.  Errors: EBUSY (a plan uses the
 * trace), ENOTFOUND (unknown id; TALP_GPU_ALL never fails this way). */
talp_gpu_status talp_gpu_reset(talp_gpu_ctx *ctx, uint64_t trace_id);

/* Device bytes the context currently holds, and its budget (host memory
 * out pointers; either may be NULL).  Library service, no passage: the
 * admission by HBM footprint that the served form applies. */
talp_gpu_status talp_gpu_memory(talp_gpu_ctx *ctx, size_t *held_bytes, size_t *budget_bytes);

/*
 * Kernel timing for benchmarks and tracing (library service, no passage).
 * While enabled, every sweep
 * launch (the pass over the records: flattening, host sums, validation) is
 * bracketed by CUDA events on the ingest stream, and so is every sort stage
 * (the kernels between the first sweep's fix-up and the re-sweep of an
 * ingest without TALP_GPU_SORTED_BY_START: run finding, the fused
 * merge-sweep, the radix passes).  talp_gpu_profile_read synchronises those
 * events, returns the totals since the last read and clears them.
 * kernel_launches counts every kernel the context launched (enabled or not).
 */
typedef struct {
    uint64_t sweep_launches;
    uint64_t sweep_records;            /* records covered by those launches */
    double sweep_ms;                   /* summed event time of those launches */
    uint64_t kernel_launches;
    uint64_t sort_launches;            /* sort stages timed */
    double sort_ms;                    /* summed event time of those stages */
} talp_gpu_profile_stats;

talp_gpu_status talp_gpu_profile(talp_gpu_ctx *ctx, int enable);
talp_gpu_status talp_gpu_profile_read(talp_gpu_ctx *ctx, talp_gpu_profile_stats *out);

/*
 * Reduction of one trace with no device allocation at all.  (The paper has
 * no counterpart: this is a service of the library, not a step of the
 * method.)
 *
 * For callers that must not call cudaMalloc or cudaFree, such as a
 * monitoring hook running inside the measured application: the application
 * or its framework's caching allocator owns the device memory (possibly all
 * of it), and an allocation or free from the hook could fail or synchronise
 * the device and stall the application's streams.  No context is needed.
 * The scratch lives in one fixed-size __device__ array of the library
 * (under 6 MiB per device, held until the process exits); the device used is
 * the calling thread's current device.
 *
 * b:        one trace with flags exactly TALP_GPU_DEVICE_PTRS |
 *           TALP_GPU_SORTED_BY_START (records in device memory, each
 *           device's records in start order); n_ranks + m must not exceed
 *           TALP_GPU_NOALLOC_MAX_UNITS, n_regions <= 8, else EINVAL.
 * out_host: n_regions metrics, one per region, in host memory.
 * The call synchronises `stream`.
 *
 * Set-up: the first call on a device looks up the scratch's device address
 * (again after a device reset).  Under CUDA's default lazy module loading
 * that first call also loads the array and the kernels' code, which the
 * driver allocates (about 6 MiB plus code): make one first call -- a trace
 * without records will do -- during set-up, before the application fills
 * the device's memory and before any stream capture.  Later calls allocate
 * nothing.
 *
 * Sharing: every call on a device uses the same array, which keeps the last
 * call's contents; each call clears what must start at zero.  Calls whose
 * GPU work overlapped would race on the array, so each call holds a lock of
 * its device from its first enqueue until its stream has finished the work,
 * also when it returns an error: calls through this library in one process
 * are serialised per device and never overlap.
 * TALP_GPU_WAIT_LIMIT (clock cycles, read at each call) bounds the
 * device-side waits as for contexts.
 * Errors: EINVAL (limits, flags, invalid or out-of-order records; out_host is
 * written and its flags say why), ETIMEDOUT, ECUDA.
 */
#define TALP_GPU_NOALLOC_MAX_UNITS 8192u
talp_gpu_status talp_gpu_reduce_noalloc(const talp_gpu_trace_batch *b, talp_gpu_metrics *out_host, void *stream);

/* Message of the last failing call on this thread ("" if none; library
 * service, no passage).  The string belongs to the library and stays valid
 * until the thread's next failing call. */
const char *talp_gpu_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TALP_GPU_H */
