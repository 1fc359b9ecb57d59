// Device-side building blocks shared by the kernels of the reducer:
// descriptors of the work, PTX wrappers for mbarriers and 1-D bulk TMA,
// warp scans/reductions of int64 values.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace talp {

constexpr int64_t NEG_INF = INT64_MIN;   // running max end before any record
constexpr uint32_t NONE = 0xFFFFFFFFu;

// validation / status bits (per segment and per trace)
constexpr uint32_t ST_BAD_END = 0x1u;      // end < start
constexpr uint32_t ST_BAD_KIND = 0x2u;     // device kind > 4 or host state > 2
constexpr uint32_t ST_UNSORTED = 0x4u;     // device starts out of order
constexpr uint32_t ST_TIMEOUT = 0x8u;      // a bounded device wait ran out

// One unit of independent work: the records of one device (a sweep with
// three running-max chains) or of one rank's host (plain clipped sums).
struct SegDesc {
    const int64_t* se;         // record 0 of the segment: {start, end}
    const uint8_t* tag;        // tag (device) or state (host) of record 0
    const uint8_t* tag_limit;  // 16-byte floor of the end of the tag array;
                               // tag bytes at or past it are read directly
    int64_t* sums;             // [R][3] accumulators of this unit
    const int64_t* win;        // [R][2] windows of the owning rank
    uint32_t* status;          // per-trace status word
    const int64_t* carry_in;   // device: {max kernel end, max memory end, last start}
                               // of earlier ingests (read only during the pass)
    int64_t* carry_out;        // device: the same after this ingest (atomic max)
    uint64_t n;                // records
    uint16_t R;                // regions
    uint8_t is_host;
    uint8_t pad[5];
};

// What one warp of the sweep publishes for the fix-up pass.
struct WarpRec {
    uint64_t head_pos;   // first virtual record index of the warp's range
    uint64_t head_end;   // end of its first portion (same segment)
    uint32_t head_seg;   // segment of head_pos (NONE: the warp had no records)
    uint32_t tail_seg;   // segment of its last portion
    int64_t head_K, head_M;  // max kernel / memory end over the first portion
    int64_t tail_K, tail_M;  // same over the last portion
};

// Device-resident descriptor of one trace, read by the finalize kernel.
struct TraceDev {
    uint64_t trace_id;
    uint32_t n, m, R;
    uint32_t pad;
    const int64_t* hsum;     // [n][R][3]  useful, offload, MPI
    const int64_t* dsum;     // [m][R][3]  kernel union, memory union, busy union
    const int64_t* hwin;     // [n][R][2]
    const int64_t* dev_rank; // [m]
    const uint32_t* status;  // trace status word
};

// Metrics record written by the finalize kernel; mirrors talp_gpu_metrics.
struct MetricsOut {
    uint64_t trace_id;
    uint32_t region, flags, n_ranks, m_devices;
    int64_t elapsed_ns, sum_useful, sum_offload, sum_mpi, max_useful_offload;
    int64_t sum_kernel, max_kernel, max_busy, sum_mem, sum_idle, sum_hidden_mem;
    double host_pe, host_mpi_pe, host_mpi_lb, host_mpi_ce, host_oe;
    double dev_pe, dev_lb, dev_ce, dev_oe;
};

// Scaling factors of one run against a reference run; mirrors talp_gpu_scaling.
struct ScaleOut {
    uint64_t trace_id;
    uint32_t region, flags, n_ranks, m_devices;
    double speedup, host_comp_scal, host_global_eff, dev_comp_scal, dev_global_eff;
};

// Host tree with threads of one region; mirrors talp_gpu_thread_metrics.
struct ThreadOut {
    uint64_t trace_id;
    uint32_t region, flags, n_procs, n_threads;
    int64_t elapsed_ns, sum_useful, sum_offload, sum_busiest, max_busiest;
    double pe, mpi_pe, mpi_lb, mpi_ce, thread_lb, oe;
};

// One (trace, region) of the thread tree; proc_off[0 .. n_procs] (device
// memory) groups the trace's host units into processes.
struct ThreadJob {
    const TraceDev* t;
    ThreadOut* out;
    const uint32_t* proc_off;
    uint32_t n_procs, region;
};

struct FinalizeJob {
    const TraceDev* t;
    MetricsOut* out;
    uint32_t region;
    uint32_t pad;
};

// (ptr, count, value) fill job for the prep kernel
struct FillJob {
    int64_t* ptr;
    uint64_t count;
    int64_t value;        // fill value; with src: 0 = copy src, 1 = add src
    const int64_t* src;
};

// SegDesc.pad[0] bits
constexpr uint8_t kSegSortable = 1;   // device segment may be sorted when found out of order
constexpr uint8_t kSegPresort = 2;    // known out of order (several streams of a raw buffer): left out
                                      // of the first sweep and sorted, then swept
constexpr uint8_t kSegGrouped = 4;    // records grouped by stream (the caller's word): its runs are
                                      // found from the stream ids before the sort stage

// Control block of the sort stage (device memory; pointers into scratch).
struct SortCtl {
    uint32_t nflag;            // flagged segments
    uint32_t max_passes;       // most radix passes any flagged segment needs
    uint64_t nrec;             // their records
    uint64_t ntile;            // their sort tiles
    uint32_t* list;            // [slots] segment index of flagged segment k
    uint64_t* rec_base;        // [slots] first record of k in the sort buffers
    uint64_t* tile_base;       // [slots + 1] first tile of k
    int64_t* mn;               // [slots] smallest start of k
    int64_t* mx;               // [slots] largest start of k
    uint32_t* hist;            // [tiles][256] digit counts
    uint64_t* offs;            // [tiles][256] output offsets
    int64_t* buf_se[2];        // ping-pong record buffers
    uint8_t* buf_tag[2];
    const uint8_t* buf_tag_limit[2];
    const int64_t* const* restore;  // [segments] sums a flagged segment restarts from (null: zero)
    const uint64_t* const* known;   // [segments] runs already known (null: none): count r, then the
                                    // r + 1 run boundaries (kRunsStride entries; r < 2: unknown)
    const uint32_t* seen_n;    // [segments] the first sweep's run log (null: none; see RunLog)
    const uint64_t* seen_pos;  // [segments][kMaxRuns]
    uint32_t* given;           // [slots] where k's runs came from (kRunsFound / kRunsKnown / kRunsSeen;
                               // the min/max pass skips k unless kRunsFound)
    uint32_t* nruns;           // [slots] descents found in k (runs - 1)
    uint64_t* runs;            // [slots][kMaxRuns + 1] run boundaries of k (sorted by the merge plan)
    uint32_t* fused;           // [slots] 1: k is a few sorted runs, merged and swept in one pass
    // fused merge-sweep (fms.cu) of the segments marked in `fused`
    uint32_t* fms_S;           // [slots] sample step of k (0: k not fused)
    uint64_t* fms_samp_base;   // [slots + 1] first sample of k in fms_samp
    uint64_t* fms_chunk_base;  // [slots + 1] first chunk of k
    uint64_t* fms_split_base;  // [slots] first entry of k's split rows in fms_split
    uint64_t* fms_sc_base;     // [slots + 1] first super-chunk of k
    int64_t* fms_samp;         // [samples] start of every sample record
    uint64_t* fms_split;       // per chunk boundary c = 0 .. nch of k: the position in each run
    uint32_t* fms_chunk_seg;   // [chunks] flagged segment of each chunk
    struct FmsChunk* fms_chunk;// [chunks] aggregate and carry of each chunk
    int64_t* fms_sc_agg;       // [super-chunks][2] largest kernel / memory end of each super-chunk
    struct FmsFix* fms_fix;    // [chunks] chunks swept again with their segment's true carry
    uint64_t fms_nsamp;        // samples over every fused segment
    uint64_t fms_nchunk;       // chunks over every fused segment
    uint64_t fms_nsc;          // super-chunks over every fused segment
    uint32_t fms_ticket;       // next super-chunk to hand out
    uint32_t fms_nfix;         // fix-up jobs
    uint32_t fms_fix_ticket;   // next fix-up job to hand out
    uint32_t n_find;           // flagged segments whose runs the min/max pass must find
};

// Per chunk of the fused merge-sweep: the largest kernel / memory end of its
// records, the carry it was swept with (the largest ends of the earlier
// chunks of its super-chunk, or the earlier ingests for a segment's first
// super-chunk) and its smallest start.
struct FmsChunk {
    int64_t aggK, aggM, LK, LM, s0;
};

// A chunk swept again with its true carry T (the fix-up adds the difference
// between the sweeps with T and with its carry L).
struct FmsFix {
    uint64_t g;                // global chunk index
    int64_t TK, TM;
};

// A flagged segment made of at most this many sorted runs (records grouped
// by stream, each stream in start order) is merged and swept in one pass
// (fms.cu) instead of being radix sorted and swept again.
constexpr int kMaxRuns = 16;
constexpr int kRunsStride = kMaxRuns + 2;   // entries of a known-runs record

// Where each device segment's start order descends, as the first sweep (and
// its fix-up, at slice boundaries) finds it: every position j >= 1 of the
// ingest's records of the segment with s_j < s_(j-1).  At most kMaxRuns - 1
// positions are kept (a segment of kMaxRuns runs); the count goes past that
// only to tell the segment is more runs than that.
struct RunLog {
    uint32_t* n;     // [segments] descents counted (null: nothing logged)
    uint64_t* pos;   // [segments][kMaxRuns] their positions, in no order
};

// SortCtl.given values: where a flagged segment's runs came from
constexpr uint32_t kRunsFound = 0;   // the min/max pass of the sort stage
constexpr uint32_t kRunsKnown = 1;   // the caller (a raw lane's streams): unchecked
constexpr uint32_t kRunsSeen = 2;    // the first sweep's run log (every pair of records checked)

// One warp (all lanes, any divergence resolved): log the descents flagged in
// `desc` at positions j of segment seg.
__device__ __forceinline__ void runlog_note(const RunLog& rl, uint32_t seg, bool desc, uint64_t j) {
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, desc);
    if (!bal) return;
    const int lane = threadIdx.x & 31;
    uint32_t base = kMaxRuns;
    if (lane == 0) {
        const uint32_t seen = *static_cast<volatile uint32_t*>(&rl.n[seg]);
        if (seen < static_cast<uint32_t>(kMaxRuns)) base = atomicAdd(&rl.n[seg], static_cast<uint32_t>(__popc(bal)));
    }
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (desc) {
        const uint32_t slot = base + __popc(bal & ((1u << lane) - 1u));
        if (slot < static_cast<uint32_t>(kMaxRuns - 1)) rl.pos[static_cast<uint64_t>(seg) * kMaxRuns + slot] = j;
    }
}
// Records per chunk of the fused merge-sweep (at most).  A segment of r runs
// is sampled every S = kFmsChunk / ((kFmsSpread + 1) r) records of each run
// and cut at every (kFmsSpread r)-th sample in merged order; a chunk then
// holds at most (kFmsSpread + 1) r S <= kFmsChunk records, about
// kFmsSpread / (kFmsSpread + 1) of that on average.  Table bounds for a
// segment of n records: at most n / S + r samples and 4 n / kFmsChunk + 2
// chunks.  kFmsSuper consecutive chunks of a segment form a super-chunk, the
// unit a CTA takes.
constexpr int kFmsChunk = 2048;
constexpr int kFmsSpread = 3;
constexpr int kFmsMinStep = kFmsChunk / ((kFmsSpread + 1) * kMaxRuns);
constexpr int kFmsSuper = 16;

// Concurrency profile: levels k = 1 .. kConcLevels of concurrently active
// records per device; one device's window and record range, and the chunks
// its records are cut into.
constexpr int kConcLevels = 8;
struct ConcDev {
    int64_t a, b;              // region window of the device's rank
    uint64_t rec0, n;          // its records in the record arrays
    uint32_t chunk0, nchunk;   // its chunks
};
struct ConcChunk {
    uint64_t rec0;             // first record
    uint32_t n;                // records
    uint32_t dev;              // device index
};

// Raw activity-record adapter: per rank its lane range and hold-back state,
// per tile of input records its source arrays and rank.
constexpr int kRawMaxDevices = 8;   // local devices per rank (buckets: device x stream)
constexpr int kRawBuckets = kRawMaxDevices * 32;
struct RawRank {
    uint64_t out0;             // first lane record (the rank's devices in order)
    uint32_t dev0;             // global index of its first device
    uint32_t D;                // its devices
    uint32_t tile0, ntile;     // its input tiles
    int64_t* last_start;       // hold-back: [D][32] last start seen per (device, stream); null: fold all
    int64_t* hold_se;          // hold-back: where its held records go (rows, tags, devices)
    uint8_t* hold_tag;
    uint8_t* hold_dev;
    uint32_t smask[kRawMaxDevices];   // hold-back: declared streams of each device
    uint32_t fresh;            // hold-back: last_start not written yet (every stream unseen)
    uint32_t pad;
};
struct RawTile {
    const int64_t* se;         // the tile's records (rows, tags, device indexes)
    const uint8_t* tag;
    const uint8_t* dev;
    uint64_t lpos;             // lane position of its first record (a rank's tiles cover its lanes in order)
    uint32_t n;                // records
    uint32_t rank;             // global rank index
};
// per (rank, bucket): its scattered records [src, src + nfold + nhold), the
// final prefix going to fold_dst and the rest to hold_dst (both relative to
// the rank's fold and hold bases)
struct RawMove {
    uint64_t src;
    uint32_t fold_dst, hold_dst;
    uint32_t nfold, nhold;
};

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: returns false when `limit` clock cycles pass first.
// Copies already issued must still land before a CTA exits: that drain
// waits with its own bound, whatever the configured limit.
constexpr int64_t kDrainWaitCycles = 4000000000LL;   // ~2 s at 2 GHz
// A negative limit reports a time-out at once: the failure path's test hook.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int64_t limit) {
    if (limit < 0) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const int64_t t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Flags published by one CTA and read by others (release / acquire at GPU scope).
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier over a subset of a CTA's warps (named barrier `id`, `threads` a
// multiple of 32); id 0 is __syncthreads.
__device__ __forceinline__ void named_bar(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// 1-D bulk copy global -> shared through the TMA unit, completing on `bar`.
// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ int64_t shfl_up64(int64_t v, int d) {
    return static_cast<int64_t>(__shfl_up_sync(0xFFFFFFFFu, static_cast<long long>(v), d));
}
__device__ __forceinline__ int64_t shfl64(int64_t v, int src) {
    return static_cast<int64_t>(__shfl_sync(0xFFFFFFFFu, static_cast<long long>(v), src));
}
__device__ __forceinline__ int64_t shfl_xor64(int64_t v, int m) {
    return static_cast<int64_t>(__shfl_xor_sync(0xFFFFFFFFu, static_cast<long long>(v), m));
}

__device__ __forceinline__ int64_t warp_sum64(int64_t v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += shfl_xor64(v, m);
    return v;
}
__device__ __forceinline__ int64_t warp_max64(int64_t v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v = max64(v, shfl_xor64(v, m));
    return v;
}

// Inclusive max-scan of two values across the warp.
__device__ __forceinline__ void warp_incl_max2(int64_t& a, int64_t& b, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t ta = shfl_up64(a, d);
        const int64_t tb = shfl_up64(b, d);
        if (lane >= d) {
            a = max64(a, ta);
            b = max64(b, tb);
        }
    }
}

__device__ __forceinline__ void atomic_add64(int64_t* p, int64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}
__device__ __forceinline__ void atomic_max64(int64_t* p, int64_t v) {
    atomicMax(reinterpret_cast<long long*>(p), static_cast<long long>(v));
}

}  // namespace talp
