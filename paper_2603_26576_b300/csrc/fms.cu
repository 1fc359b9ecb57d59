// Fused merge-sweep: the flattening of Sec. 4.2 over device segments made of
// a few sorted runs laid end to end (records grouped by stream, each stream
// in start order -- the order per-stream activity buffers deliver).
//
// The union arithmetic needs each device's records in start order.  Instead
// of materialising a sorted copy and sweeping it again, the records are
// merged chunk by chunk in shared memory and swept there, so they cross HBM
// once.
//
// Order: records are taken in the total order (start, run, position), a
// strict order in which equal starts are resolved by run; unions do not
// depend on how equal starts are ordered.
//
// Chunks: every S-th record of each run is a sample (S = kFmsChunk /
// ((kFmsSpread + 1) r) for r runs) and every (kFmsSpread r)-th sample in
// merged order a splitter; chunk c of a segment holds the records between
// splitters c and c + 1.  Each run contributes a contiguous range to a
// chunk, at most (x + 1) S records when x of its samples fall in the chunk,
// and a chunk holds kFmsSpread r samples, so a chunk has at most
// (kFmsSpread + 1) r S <= kFmsChunk records.  The positions of a splitter in
// the other runs follow from the samples by a binary search inside one
// sample block.
//
// Sweep (one CTA per super-chunk of kFmsSuper consecutive chunks of a
// segment at a time; a producer warp and 8 consumer warps):
//  - the producer stages each run's range of a chunk in shared memory with
//    1-D bulk copies (cp.async.bulk) completing on the stage's mbarrier (it
//    never waits for its copies; one stage, so that three CTAs fit on an SM
//    and hide each other's copies and barriers);
//  - the consumers take the chunk's largest kernel and memory ends (its
//    aggregate) and validate its records, rank every record by merge path
//    (its position in its run plus the number of records of every other run
//    before it) and sweep the merged order with the arithmetic of the
//    streaming sweep (chains K, M, all; new pieces [max(s, P), e); the region
//    windows classified once per chunk), the carry into the chunk being the
//    largest ends of the earlier chunks of its super-chunk (for a segment's
//    first super-chunk, of the earlier ingests too).
// No CTA waits for another.  A super-chunk's true carry (the largest ends of
// everything before it) is known once all are swept: a scan over the
// super-chunks' aggregates gives it, and the leading chunks of a super-chunk
// whose carry was too small are swept again (fix-up) with both carries, the
// difference added to the sums.  Only records starting below the true carry
// are affected, so that is usually one chunk per super-chunk.
#include "kernels.h"
#include "sweep_core.cuh"

namespace talp {

namespace {

constexpr int kFmsConsumers = 8;                   // consumer warps
constexpr int kFmsThreads = 32 * (kFmsConsumers + 1);
constexpr int kFmsCT = 32 * kFmsConsumers;         // consumer threads
constexpr int kFmsItems = kFmsChunk / kFmsCT;      // records per consumer thread (at most)
constexpr int kFmsStages = 1;                     // 3 CTAs per SM: 72 KB, 72 registers
constexpr int kFmsTagBytes = kFmsChunk + 32 * kMaxRuns;
constexpr int kRmax = 8;                           // regions per trace (at most)

// The fields of a chunk's segment descriptor the consumers use, copied by
// the producer (one 8-byte word per lane) so that the consumers find them in
// shared memory instead of behind two dependent global loads.
struct SegCopy {
    int64_t win[2 * kRmax];        // region windows
    int64_t cin[3];                // carry_in: largest kernel / memory end, last start of earlier ingests
    int64_t* sums;
    uint32_t* status;
    int64_t* cout;                 // carry_out
    int64_t R;                     // regions
    int64_t seg;                   // segment index (ctl->list[k])
    const uint8_t* tag;
    const int64_t* se;
};
constexpr int kSegCopyWords = 2 * kRmax + 10;
static_assert(sizeof(SegCopy) == 8 * kSegCopyWords, "one 8-byte word per field");
static_assert(kSegCopyWords <= 32, "one word per producer lane");

// per-chunk description written by the producer for the consumers
struct ChunkMeta {
    uint64_t g;                    // global chunk index
    uint64_t sc;                   // its super-chunk (main pass)
    uint32_t k, c, nr, n, valid;
    uint32_t first, last, seg_first;   // first / last chunk of its super-chunk; super-chunk 0 of its segment
    uint32_t given;                // the segment's runs came from the caller, unchecked (kRunsKnown)
    int64_t LK, LM;                // fix-up: the carry it was swept with
    int64_t TK, TM;                // fix-up: the true carry
    uint32_t roff[kMaxRuns + 1];   // staging row offset of each run's range (prefix)
    uint32_t tpos[kMaxRuns];       // tag-area index of each range's first tag
    uint32_t direct[kMaxRuns];     // first range index whose tag the bulk copy does not cover
    uint64_t lo[kMaxRuns];         // position of each range in its run's segment
    SegCopy sd;                    // its segment's descriptor fields
};

struct __align__(16) FmsStage {
    longlong2 rows[kFmsChunk];
    uint8_t tags[kFmsTagBytes];    // per run: the 16-byte aligned superset of its tags
};

struct FmsShared {
    FmsStage st[kFmsStages];
    // chunk descriptions, two deep: the consumers hand the stage back as soon
    // as they no longer read its rows and tags (after the chunk's aggregate
    // on the 32-bit path), and the producer then fills the stage and the
    // other description while they merge and sweep
    ChunkMeta meta[2];
    // the chunk the consumers work on: merged order (two index buffers for
    // the merge rounds), and every record's tag, start and end in staging
    // order (start and end as 32-bit offsets from the chunk's smallest start,
    // when its span allows; the merge rounds of that case carry the keys)
    uint16_t ix[2][kFmsChunk];
    uint32_t key[2][kFmsChunk];
    uint32_t end32[kFmsChunk];
    uint8_t tagc[kFmsChunk];
    uint64_t full[kFmsStages], empty[kFmsStages];
    int64_t red64[kFmsConsumers][4];
    uint32_t red32[kFmsConsumers][4];
    int64_t win[2 * kRmax];
    int64_t LK, LM;                // main pass: the carry into the next chunk of the super-chunk
    int64_t scK, scM;              // main pass: the super-chunk's aggregate so far
    uint32_t bad;
    uint32_t tmo;                  // consumer waits that ran out (never reset)
};

__device__ __forceinline__ void cbar() { named_bar(1, kFmsCT); }

__device__ __forceinline__ uint32_t fms_step(uint32_t nr) {
    return static_cast<uint32_t>(kFmsChunk) / static_cast<uint32_t>((kFmsSpread + 1) * nr);
}

// number of samples of a run of len records
__device__ __forceinline__ uint64_t n_samples(uint64_t len, uint32_t S) { return (len + S - 1) / S; }

// ------------------------------------------------------------------ plan
// One CTA: sample step, sample / chunk / split-row / super-chunk bases of
// every fused segment (block-wide scans), split rows 0 and nch (the runs'
// ends), the chunk-0 entries, and the totals.
__global__ void __launch_bounds__(1024) fms_plan_kernel(SortCtl* ctl) {
    __shared__ uint64_t s_a[32], s_b[32], s_c[32], s_d[32];
    __shared__ uint64_t s_base[4];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid < 4) s_base[tid] = 0;
    __syncthreads();
    const uint32_t nflag = ctl->nflag;
    for (uint32_t c0 = 0; c0 < nflag; c0 += blockDim.x) {
        const uint32_t k = c0 + tid;
        uint64_t ns = 0, nch = 0, nsp = 0, nsc = 0;
        uint32_t nr = 0, S = 0;
        if (k < nflag && ctl->fused[k]) {
            nr = ctl->nruns[k] + 1;
            S = fms_step(nr);
            const uint64_t* runs = ctl->runs + static_cast<uint64_t>(k) * (kMaxRuns + 1);
            for (uint32_t q = 0; q < nr; ++q) ns += n_samples(runs[q + 1] - runs[q], S);
            const uint64_t per = static_cast<uint64_t>(kFmsSpread) * nr;
            nch = (ns + per - 1) / per;
            nsp = (nch + 1) * nr;
            nsc = (nch + kFmsSuper - 1) / kFmsSuper;
        }
        uint64_t wa = ns, wb = nch, wc = nsp, wd = nsc;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
            const uint64_t a = __shfl_up_sync(0xFFFFFFFFu, wa, dd);
            const uint64_t b = __shfl_up_sync(0xFFFFFFFFu, wb, dd);
            const uint64_t c = __shfl_up_sync(0xFFFFFFFFu, wc, dd);
            const uint64_t e = __shfl_up_sync(0xFFFFFFFFu, wd, dd);
            if (lane >= dd) {
                wa += a;
                wb += b;
                wc += c;
                wd += e;
            }
        }
        if (lane == 31) {
            s_a[wid] = wa;
            s_b[wid] = wb;
            s_c[wid] = wc;
            s_d[wid] = wd;
        }
        __syncthreads();
        uint64_t pa = 0, pb = 0, pc = 0, pd = 0;
        for (int w = 0; w < wid; ++w) {
            pa += s_a[w];
            pb += s_b[w];
            pc += s_c[w];
            pd += s_d[w];
        }
        if (k < nflag) {
            const uint64_t sb = s_base[0] + pa + wa - ns, cb = s_base[1] + pb + wb - nch;
            const uint64_t pb0 = s_base[2] + pc + wc - nsp, scb = s_base[3] + pd + wd - nsc;
            ctl->fms_S[k] = S;
            ctl->fms_samp_base[k] = sb;
            ctl->fms_chunk_base[k] = cb;
            ctl->fms_split_base[k] = pb0;
            ctl->fms_sc_base[k] = scb;
            if (nr) {
                const uint64_t* runs = ctl->runs + static_cast<uint64_t>(k) * (kMaxRuns + 1);
                for (uint32_t q = 0; q < nr; ++q) {
                    ctl->fms_split[pb0 + q] = runs[q];                 // chunk 0 starts at every run's start
                    ctl->fms_split[pb0 + nch * nr + q] = runs[q + 1];  // the last chunk ends at every run's end
                }
                ctl->fms_chunk_seg[cb] = k;
            }
        }
        __syncthreads();
        if (tid == blockDim.x - 1) {
            s_base[0] += pa + wa;
            s_base[1] += pb + wb;
            s_base[2] += pc + wc;
            s_base[3] += pd + wd;
        }
        __syncthreads();
    }
    if (tid == 0) {
        ctl->fms_samp_base[nflag] = s_base[0];
        ctl->fms_chunk_base[nflag] = s_base[1];
        ctl->fms_sc_base[nflag] = s_base[3];
        ctl->fms_nsamp = s_base[0];
        ctl->fms_nchunk = s_base[1];
        ctl->fms_nsc = s_base[3];
        ctl->fms_ticket = 0;
        ctl->fms_nfix = 0;
        ctl->fms_fix_ticket = 0;
    }
}

// index of the last entry of base[0 .. n) that is <= x (base non-decreasing)
__device__ __forceinline__ uint32_t upper_index(const uint64_t* base, uint32_t n, uint64_t x) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (base[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// run q and block b of local sample l of a fused segment
__device__ __forceinline__ void sample_run(const uint64_t* runs, uint32_t nr, uint32_t S, uint64_t l, uint32_t& q,
                                           uint64_t& b) {
    uint64_t acc = 0;
    q = 0;
    for (;;) {
        const uint64_t t = n_samples(runs[q + 1] - runs[q], S);
        if (l < acc + t || q + 1 == nr) break;
        acc += t;
        ++q;
    }
    b = l - acc;
}

// ---------------------------------------------------------------- samples
__global__ void __launch_bounds__(256) fms_sample_kernel(const SegDesc* __restrict__ segs, SortCtl* ctl) {
    const uint64_t total = ctl->fms_nsamp;
    for (uint64_t g = blockIdx.x * 256ull + threadIdx.x; g < total; g += gridDim.x * 256ull) {
        const uint32_t k = upper_index(ctl->fms_samp_base, ctl->nflag, g);
        const uint32_t nr = ctl->nruns[k] + 1, S = ctl->fms_S[k];
        const uint64_t* runs = ctl->runs + static_cast<uint64_t>(k) * (kMaxRuns + 1);
        uint32_t q;
        uint64_t b;
        sample_run(runs, nr, S, g - ctl->fms_samp_base[k], q, b);
        const SegDesc& d = segs[ctl->list[k]];
        ctl->fms_samp[g] = d.se[2 * (runs[q] + b * S)];
    }
}

// ------------------------------------------------------------------ split
// One thread per sample: its merged rank among the segment's samples (its
// block index plus the samples of every other run before it in the total
// order); a sample of rank c * kFmsSpread * r (c >= 1) is the splitter of
// chunk c and gives the chunk's first position in every run.
__global__ void __launch_bounds__(256) fms_split_kernel(const SegDesc* __restrict__ segs, SortCtl* ctl) {
    const uint64_t total = ctl->fms_nsamp;
    for (uint64_t g = blockIdx.x * 256ull + threadIdx.x; g < total; g += gridDim.x * 256ull) {
        const uint32_t k = upper_index(ctl->fms_samp_base, ctl->nflag, g);
        const uint32_t nr = ctl->nruns[k] + 1, S = ctl->fms_S[k];
        const uint64_t* runs = ctl->runs + static_cast<uint64_t>(k) * (kMaxRuns + 1);
        const uint64_t sb = ctl->fms_samp_base[k];
        uint32_t q;
        uint64_t b;
        sample_run(runs, nr, S, g - sb, q, b);
        const int64_t key = ctl->fms_samp[g];
        uint64_t cnt[kMaxRuns];
        uint64_t rank = b;
        uint64_t first = 0;
        for (uint32_t p = 0; p < nr; ++p) {
            const uint64_t t = n_samples(runs[p + 1] - runs[p], S);
            uint64_t c = 0;
            if (p != q) {
                // samples of run p before (key, q): key' <= key for p < q, key' < key for p > q
                const int64_t* sp = ctl->fms_samp + sb + first;
                uint64_t lo = 0, hi = t;
                while (lo < hi) {
                    const uint64_t mid = (lo + hi) >> 1;
                    const int64_t v = sp[mid];
                    if (p < q ? v <= key : v < key) lo = mid + 1; else hi = mid;
                }
                c = lo;
                rank += c;
            }
            cnt[p] = c;
            first += t;
        }
        const uint64_t per = static_cast<uint64_t>(kFmsSpread) * nr;
        if (rank == 0 || rank % per != 0) continue;
        const uint64_t ch = rank / per;
        const SegDesc& d = segs[ctl->list[k]];
        uint64_t* row = ctl->fms_split + ctl->fms_split_base[k] + ch * nr;
        for (uint32_t p = 0; p < nr; ++p) {
            uint64_t pos;
            if (p == q) {
                pos = runs[q] + b * S;
            } else if (cnt[p] == 0) {
                pos = runs[p];
            } else {
                // records of run p before the splitter: the first (cnt - 1) S + 1
                // precede it, none from cnt S on; the boundary lies in between
                uint64_t lo = runs[p] + (cnt[p] - 1) * S + 1;
                uint64_t hi = runs[p] + cnt[p] * S;
                if (hi > runs[p + 1]) hi = runs[p + 1];
                while (lo < hi) {
                    const uint64_t mid = (lo + hi) >> 1;
                    const int64_t v = d.se[2 * mid];
                    if (p < q ? v <= key : v < key) lo = mid + 1; else hi = mid;
                }
                pos = lo;
            }
            row[p] = pos;
        }
        ctl->fms_chunk_seg[ctl->fms_chunk_base[k] + ch] = k;
    }
}

// -------------------------------------------------------------- consumers

// CTA-wide (consumer) sums of three values below 2^51 per thread; every
// consumer thread gets the totals.
__device__ __forceinline__ void cta_sum3(FmsShared& sh, int ct, uint64_t a, uint64_t b, uint64_t c, int64_t& ta,
                                         int64_t& tb, int64_t& tc) {
    const int lane = ct & 31, w = ct >> 5;
    const int64_t x = warp_sum_u64_small(a), y = warp_sum_u64_small(b), z = warp_sum_u64_small(c);
    if (lane == 0) {
        sh.red64[w][0] = x;
        sh.red64[w][1] = y;
        sh.red64[w][2] = z;
    }
    cbar();
    ta = tb = tc = 0;
#pragma unroll
    for (int q = 0; q < kFmsConsumers; ++q) {
        ta += sh.red64[q][0];
        tb += sh.red64[q][1];
        tc += sh.red64[q][2];
    }
    cbar();
}

// Records per consumer thread for a chunk of n records.
__device__ __forceinline__ uint32_t items_for(uint32_t n) { return (n + kFmsCT - 1) / kFmsCT; }

// Merged order of a chunk's staged records: ceil(log2 r) rounds of pairwise
// merges of adjacent groups of runs, each thread producing E consecutive
// outputs of a round by merge path (a binary search for its first output,
// then one comparison per output; ties from the left group, so the order is
// (start, run, position)).  Round 0 reads the staged rows in place; each round
// writes staging indices to sh.ix[round & 1].  Returns the buffer holding
// the final order.  Ends with a consumer barrier.
__device__ __forceinline__ int merge_rounds(FmsShared& sh, const FmsStage& S, const ChunkMeta& M, int ct, uint32_t E) {
    const uint32_t n = M.n, nr = M.nr;
    uint32_t width = 1;   // runs per group entering the round
    int round = 0;
    while (width < nr) {
        const uint16_t* in = sh.ix[(round + 1) & 1];   // the previous round's output (unused in round 0)
        uint16_t* out = sh.ix[round & 1];
        const uint32_t o0 = static_cast<uint32_t>(ct) * E;
        const uint32_t o1 = min(n, o0 + E);
        uint32_t o = o0;
        while (o < o1) {
            // the pair of groups holding output o: groups [g, g + width) and [g + width, g + 2 width)
            uint32_t g = 0;
            while (M.roff[min(g + 2 * width, nr)] <= o) g += 2 * width;
            const uint32_t a0 = M.roff[g], a1 = M.roff[min(g + width, nr)], b1 = M.roff[min(g + 2 * width, nr)];
            const uint32_t la = a1 - a0, lb = b1 - a1;
            const uint32_t l = o - a0;
            // key of the x-th record of the left / right group
            auto keyA = [&](uint32_t x) -> int64_t { return S.rows[round ? in[a0 + x] : a0 + x].x; };
            auto keyB = [&](uint32_t x) -> int64_t { return S.rows[round ? in[a1 + x] : a1 + x].x; };
            uint32_t lo = l > lb ? l - lb : 0u, hi = l < la ? l : la;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (keyA(mid) <= keyB(l - mid - 1)) lo = mid + 1; else hi = mid;
            }
            uint32_t i = lo, j = l - lo;
            const uint32_t stop = min(o1, b1);
            int64_t ka = i < la ? keyA(i) : INT64_MAX, kb = j < lb ? keyB(j) : INT64_MAX;
            for (; o < stop; ++o) {
                const bool takeA = j >= lb || (i < la && ka <= kb);
                uint32_t src;
                if (takeA) {
                    src = round ? in[a0 + i] : a0 + i;
                    ++i;
                    ka = i < la ? keyA(i) : INT64_MAX;
                } else {
                    src = round ? in[a1 + j] : a1 + j;
                    ++j;
                    kb = j < lb ? keyB(j) : INT64_MAX;
                }
                out[o] = static_cast<uint16_t>(src);
            }
        }
        cbar();
        width *= 2;
        ++round;
    }
    return (round - 1) & 1;
}

// The 32-bit merge of a chunk (span within 2^32 ns of its smallest start):
// the same pairwise merge-path rounds over (key, staging index) pairs held in
// compact arrays, key = start offset.  Round 0 reads sh.key[0] in staging
// order (index = position); each round but the last writes key[(r + 1) & 1]
// and ix[(r + 1) & 1]; the last round (one pair: everything) writes its
// outputs -- thread ct's E consecutive positions of the merged order, the
// same block the sweep gives the thread -- straight into the thread's
// registers: start and end offsets and tag.  cnt: records of the thread.
__device__ __forceinline__ void merge32(FmsShared& sh, const ChunkMeta& M, int ct, uint32_t E, int cnt,
                                        uint32_t (&sr)[kFmsItems], uint32_t (&er)[kFmsItems],
                                        uint32_t (&tg)[kFmsItems]) {
    const uint32_t n = M.n, nr = M.nr;
    uint32_t width = 1;   // runs per group entering the round
    int r = 0;
    for (; 2 * width < nr; width *= 2, ++r) {
        const uint32_t* kin = sh.key[r & 1];
        const uint16_t* iin = sh.ix[r & 1];
        uint32_t* kout = sh.key[(r + 1) & 1];
        uint16_t* iout = sh.ix[(r + 1) & 1];
        const uint32_t o0 = static_cast<uint32_t>(ct) * E;
        const uint32_t o1 = min(n, o0 + E);
        uint32_t o = o0;
        while (o < o1) {
            uint32_t g = 0;
            while (M.roff[min(g + 2 * width, nr)] <= o) g += 2 * width;
            const uint32_t a0 = M.roff[g], a1 = M.roff[min(g + width, nr)], b1 = M.roff[min(g + 2 * width, nr)];
            const uint32_t la = a1 - a0, lb = b1 - a1;
            const uint32_t l = o - a0;
            uint32_t lo = l > lb ? l - lb : 0u, hi = l < la ? l : la;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (kin[a0 + mid] <= kin[a1 + l - mid - 1]) lo = mid + 1; else hi = mid;
            }
            uint32_t i = lo, j = l - lo;
            const uint32_t stop = min(o1, b1);
            uint32_t ka = i < la ? kin[a0 + i] : 0xFFFFFFFFu, kb = j < lb ? kin[a1 + j] : 0xFFFFFFFFu;
            for (; o < stop; ++o) {
                const bool takeA = ka <= kb;   // an exhausted run reads as the sentinel
                const uint32_t at = takeA ? a0 + i : a1 + j;
                kout[o] = takeA ? ka : kb;
                iout[o] = r ? iin[at] : static_cast<uint16_t>(at);
                // the taken run's next key, at + 1, unless that run is used up:
                // one predicated load, no divergent branch
                i += takeA ? 1u : 0u;
                j += takeA ? 0u : 1u;
                const uint32_t nx = at + 1 < (takeA ? a1 : b1) ? kin[at + 1] : 0xFFFFFFFFu;
                ka = takeA ? nx : ka;
                kb = takeA ? kb : nx;
            }
        }
        cbar();
    }
    // the last round: groups [0, width) and [width, nr) of runs
    const uint32_t* kin = sh.key[r & 1];
    const uint16_t* iin = sh.ix[r & 1];
    const uint32_t a1 = M.roff[min(width, nr)];
    const uint32_t la = a1, lb = n - a1;
    const uint32_t l = static_cast<uint32_t>(ct) * E;
    uint32_t i = 0, j = 0;
    if (cnt > 0) {
        uint32_t lo = l > lb ? l - lb : 0u, hi = l < la ? l : la;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (kin[mid] <= kin[a1 + l - mid - 1]) lo = mid + 1; else hi = mid;
        }
        i = lo;
        j = l - lo;
    }
    uint32_t ka = i < la ? kin[i] : 0xFFFFFFFFu, kb = j < lb ? kin[a1 + j] : 0xFFFFFFFFu;
#pragma unroll
    for (int q = 0; q < kFmsItems; ++q) {
        if (q < cnt) {
            const bool takeA = ka <= kb;   // an exhausted run reads as the sentinel
            const uint32_t at = takeA ? i : a1 + j;
            const uint32_t x = r ? iin[at] : at;
            sr[q] = takeA ? ka : kb;
            er[q] = sh.end32[x];
            tg[q] = sh.tagc[x];
            i += takeA ? 1u : 0u;
            j += takeA ? 0u : 1u;
            const uint32_t nx = at + 1 < (takeA ? a1 : n) ? kin[at + 1] : 0xFFFFFFFFu;
            ka = takeA ? nx : ka;
            kb = takeA ? kb : nx;
        } else {
            sr[q] = er[q] = tg[q] = 0;
        }
    }
}

__device__ __forceinline__ void add_sums(int64_t* p, int64_t a, int64_t b, int64_t c) {
    if (a) atomic_add64(p + 0, a);
    if (b) atomic_add64(p + 1, b);
    if (c) atomic_add64(p + 2, c);
}

// The exact int64 sweep of a chunk in merged order (a chunk spanning 2^32 ns
// or more, or a carry that far ahead): per thread its records, carries by a
// CTA-wide exclusive max-scan, then the clipped pieces of every region,
// added to sums with the given sign.
__device__ void sweep64(FmsShared& sh, const FmsStage& S, const ChunkMeta& M, const uint16_t* perm, int ct, uint32_t E,
                        int R, int64_t cK, int64_t cM, int64_t* sums, int64_t sign) {
    const int lane = ct & 31, w = ct >> 5;
    const uint32_t p0 = static_cast<uint32_t>(ct) * E;
    const int cnt = p0 < M.n ? static_cast<int>(min(E, M.n - p0)) : 0;
    int64_t aK = NEG_INF, aM = NEG_INF;
    for (int i = 0; i < cnt; ++i) {
        const longlong2 v = S.rows[perm[p0 + i]];
        if ((sh.tagc[perm[p0 + i]] >> 5) == 0) aK = max64(aK, v.y); else aM = max64(aM, v.y);
    }
    int64_t iK = aK, iM = aM;
    warp_incl_max2(iK, iM, lane);
    if (lane == 31) {
        sh.red64[w][0] = iK;
        sh.red64[w][1] = iM;
    }
    cbar();
    int64_t xK = shfl_up64(iK, 1), xM = shfl_up64(iM, 1);
    if (lane == 0) xK = xM = NEG_INF;
    for (int q = 0; q < w; ++q) {
        xK = max64(xK, sh.red64[q][0]);
        xM = max64(xM, sh.red64[q][1]);
    }
    cbar();
    xK = max64(xK, cK);
    xM = max64(xM, cM);
    for (int r = 0; r < R; ++r) {
        const int64_t a = sh.win[2 * r], b = sh.win[2 * r + 1];
        int64_t Kp = xK, Mp = xM, s0 = 0, s1 = 0, s2 = 0;
        for (int i = 0; i < cnt; ++i) {
            const longlong2 v = S.rows[perm[p0 + i]];
            const bool isK = (sh.tagc[perm[p0 + i]] >> 5) == 0;
            const int64_t pA = max64(max64(v.x, max64(Kp, Mp)), a);
            const int64_t pO = max64(max64(v.x, isK ? Kp : Mp), a);
            const int64_t e = min64(v.y, b);
            s2 += max64(e - pA, 0);
            const int64_t lO = max64(e - pO, 0);
            if (isK) {
                s0 += lO;
                Kp = max64(Kp, v.y);
            } else {
                s1 += lO;
                Mp = max64(Mp, v.y);
            }
        }
        s0 = warp_sum64(s0);
        s1 = warp_sum64(s1);
        s2 = warp_sum64(s2);
        if (lane == 0) {
            sh.red64[w][0] = s0;
            sh.red64[w][1] = s1;
            sh.red64[w][2] = s2;
        }
        cbar();
        if (ct == 0) {
            int64_t t0 = 0, t1 = 0, t2 = 0;
            for (int q = 0; q < kFmsConsumers; ++q) {
                t0 += sh.red64[q][0];
                t1 += sh.red64[q][1];
                t2 += sh.red64[q][2];
            }
            add_sums(sums + 3 * r, sign * t0, sign * t1, sign * t2);
        }
        cbar();
    }
}

// The 32-bit sweep of a chunk in merged order (records, carries and span
// within 2^32 ns of s0): the registers hold the thread's records; pieces with
// carries (cK, cM) added to sums with the given sign.
__device__ __forceinline__ void sweep32(FmsShared& sh, int64_t s0, int64_t spanHi, int ct, int cnt, int R,
                                        const uint32_t (&sr)[kFmsItems], const uint32_t (&er)[kFmsItems],
                                        const uint32_t (&tg)[kFmsItems], uint32_t bK, uint32_t bM, int64_t cK,
                                        int64_t cM, int64_t* sums, int64_t sign) {
    const int lane = ct & 31, cw = ct >> 5;
    // CTA-wide exclusive max-scan of the threads' largest ends
    uint32_t iK = bK, iM = bM;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, iK, dd);
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, iM, dd);
        if (lane >= dd) {
            iK = umax(iK, x);
            iM = umax(iM, y);
        }
    }
    if (lane == 31) {
        sh.red32[cw][0] = iK;
        sh.red32[cw][1] = iM;
    }
    cbar();
    uint32_t xK = __shfl_up_sync(0xFFFFFFFFu, iK, 1), xM = __shfl_up_sync(0xFFFFFFFFu, iM, 1);
    if (lane == 0) xK = xM = 0u;
    for (int q = 0; q < cw; ++q) {
        xK = umax(xK, sh.red32[q][0]);
        xM = umax(xM, sh.red32[q][1]);
    }
    xK = umax(xK, cK <= s0 ? 0u : static_cast<uint32_t>(cK - s0));
    xM = umax(xM, cM <= s0 ? 0u : static_cast<uint32_t>(cM - s0));
    uint32_t s1 = 0, s2 = 0, s3 = 0;
    pieces32<kFmsItems, false>(sr, er, tg, cnt, xK, xM, 0u, 0xFFFFFFFFu, s1, s2, s3);
    int64_t t0, t1, t2;
    cta_sum3(sh, ct, s1, s2, s3, t0, t1, t2);   // its barriers also end every read of red32
    for (int r = 0; r < R; ++r) {
        const int64_t a = sh.win[2 * r], b = sh.win[2 * r + 1];
        if (a <= s0 && spanHi <= b) {
            if (ct == 0) add_sums(sums + 3 * r, sign * t0, sign * t1, sign * t2);
        } else if (!(spanHi <= a || s0 >= b)) {
            uint32_t k1 = 0, k2 = 0, k3 = 0;
            pieces32<kFmsItems, false>(sr, er, tg, cnt, xK, xM, rel_sat(a, s0), rel_sat(b, s0), k1, k2, k3);
            int64_t c0, c1, c2;
            cta_sum3(sh, ct, k1, k2, k3, c0, c1, c2);
            if (ct == 0) add_sums(sums + 3 * r, sign * c0, sign * c1, sign * c2);
        }
    }
}

// ------------------------------------------------------------------ kernel
// FIX = false: every chunk of every fused segment, super-chunk by
// super-chunk, with the carry of its super-chunk.  FIX = true: the fix-up
// jobs, each chunk swept with its true carry T and with its carry L, the
// difference added.
template <bool FIX>
__global__ void __launch_bounds__(kFmsThreads, 3)
    fms_kernel(const SegDesc* __restrict__ segs, SortCtl* ctl, uint32_t* __restrict__ seg_flags,
               uint32_t* __restrict__ gstatus, int64_t wait_limit) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    FmsShared& sh = *reinterpret_cast<FmsShared*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (FIX ? ctl->fms_nfix == 0 : ctl->fms_nchunk == 0) return;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kFmsStages; ++s) {
            mbar_init(&sh.full[s], 1);
            mbar_init(&sh.empty[s], 1);
        }
        sh.tmo = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == 0) {
        // ---------------------------------------------------- producer
        // Chunk descriptors and bulk copies only: the producer never waits for
        // its copies, so it runs up to kFmsStages chunks ahead of the consumers.
        uint64_t g = 0, g_end = 0;   // chunks of the current super-chunk (main pass)
        uint64_t sc = 0, scb = 0;
        uint32_t k = 0, nr = 0;
        uint64_t split0 = 0, cb = 0, lo_next = 0;
        const int64_t* dse = nullptr;
        const uint8_t* dtag = nullptr;
        uintptr_t lim = 0;
        uint64_t dn = 0;
        uint32_t given = 0;
        bool first = false;
        int64_t sdw = 0;   // this lane's word of the segment copy (SegCopy order)
        for (uint32_t it = 0;; ++it) {
            const int s = static_cast<int>(it % kFmsStages);
            if (it >= static_cast<uint32_t>(kFmsStages)) {
                bool ok = true;
                if (lane == 0) ok = mbar_wait_bounded(&sh.empty[s], ((it / kFmsStages) - 1) & 1u, wait_limit);
                if (!__shfl_sync(0xFFFFFFFFu, ok, 0)) {
                    if (lane == 0) atomicOr(gstatus, ST_TIMEOUT);
                    break;
                }
            }
            FmsStage& S = sh.st[s];
            ChunkMeta& MT = sh.meta[it & 1];
            // ---- the next chunk, and its segment's descriptor when it changes
            bool more = true, fresh = false;
            int64_t TK = NEG_INF, TM = NEG_INF, LK = NEG_INF, LM = NEG_INF;
            if (FIX) {
                uint32_t j = 0;
                if (lane == 0) j = atomicAdd(&ctl->fms_fix_ticket, 1u);
                j = __shfl_sync(0xFFFFFFFFu, j, 0);
                if (j >= ctl->fms_nfix) {
                    more = false;
                } else {
                    const FmsFix fx = ctl->fms_fix[j];
                    g = fx.g;
                    TK = fx.TK;
                    TM = fx.TM;
                    LK = ctl->fms_chunk[g].LK;
                    LM = ctl->fms_chunk[g].LM;
                    k = ctl->fms_chunk_seg[g];
                    fresh = true;
                }
            } else if (g == g_end) {
                uint32_t j = 0;
                if (lane == 0) j = atomicAdd(&ctl->fms_ticket, 1u);
                j = __shfl_sync(0xFFFFFFFFu, j, 0);
                if (j >= ctl->fms_nsc) {
                    more = false;
                } else {
                    sc = j;
                    k = upper_index(ctl->fms_sc_base, ctl->nflag, sc);
                    scb = ctl->fms_sc_base[k];
                    const uint64_t ce = ctl->fms_chunk_base[k + 1];
                    cb = ctl->fms_chunk_base[k];
                    g = cb + (sc - scb) * kFmsSuper;
                    g_end = min(g + static_cast<uint64_t>(kFmsSuper), ce);
                    fresh = true;
                    first = true;
                }
            }
            if (!more) {
                if (lane == 0) {
                    MT.valid = 0;
                    mbar_arrive(&sh.full[s]);
                }
                break;
            }
            if (fresh) {
                const uint32_t sid = ctl->list[k];
                const SegDesc& d = segs[sid];
                if (lane < 2 * kRmax) sdw = lane < 2 * static_cast<int>(d.R) ? d.win[lane] : 0;
                else if (lane < 2 * kRmax + 3) sdw = d.carry_in[lane - 2 * kRmax];
                else if (lane == 2 * kRmax + 3) sdw = reinterpret_cast<int64_t>(d.sums);
                else if (lane == 2 * kRmax + 4) sdw = reinterpret_cast<int64_t>(d.status);
                else if (lane == 2 * kRmax + 5) sdw = reinterpret_cast<int64_t>(d.carry_out);
                else if (lane == 2 * kRmax + 6) sdw = d.R;
                else if (lane == 2 * kRmax + 7) sdw = sid;
                else if (lane == 2 * kRmax + 8) sdw = reinterpret_cast<int64_t>(d.tag);
                else if (lane == 2 * kRmax + 9) sdw = reinterpret_cast<int64_t>(d.se);
                dse = d.se;
                dtag = d.tag;
                lim = reinterpret_cast<uintptr_t>(d.tag_limit);
                dn = d.n;
                nr = ctl->nruns[k] + 1;
                split0 = ctl->fms_split_base[k];
                cb = ctl->fms_chunk_base[k];
                given = ctl->given[k] == kRunsKnown;
            }
            const uint32_t c = static_cast<uint32_t>(g - cb);
            const uint64_t* row = ctl->fms_split + split0 + static_cast<uint64_t>(c) * nr;
            uint64_t lo = 0, hi = 0;
            if (lane < static_cast<int>(nr)) {
                lo = fresh ? row[lane] : lo_next;   // a chunk starts where the previous one ended
                hi = row[nr + lane];
            }
            lo_next = hi;
            const uint32_t len = static_cast<uint32_t>(hi - lo);
            const uintptr_t A = reinterpret_cast<uintptr_t>(dtag + lo);
            const uintptr_t tlo = A & ~static_cast<uintptr_t>(15);
            uintptr_t thi = (A + len + 15) & ~static_cast<uintptr_t>(15);
            if (thi > lim) thi = lim;
            const uint32_t tb = (len && thi > tlo) ? static_cast<uint32_t>(thi - tlo) : 0u;
            const uint32_t tsz = len ? static_cast<uint32_t>(((A & 15u) + len + 15u) & ~15u) : 0u;
            const uint32_t direct = lim > A ? static_cast<uint32_t>(min(static_cast<uint64_t>(lim - A),
                                                                       static_cast<uint64_t>(len))) : 0u;
            // exclusive scans of the range lengths and tag-area sizes over the runs
            uint32_t ro = len, to = tsz;
#pragma unroll
            for (int dd = 1; dd < 32; dd <<= 1) {
                const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, ro, dd);
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, to, dd);
                if (lane >= dd) {
                    ro += x;
                    to += y;
                }
            }
            const uint32_t n_tot = __shfl_sync(0xFFFFFFFFu, ro, 31);
            const uint32_t t_tot = __shfl_sync(0xFFFFFFFFu, to, 31);
            ro -= len;
            to -= tsz;
            uint32_t bytes = len * 16u + tb;
#pragma unroll
            for (int m = 16; m > 0; m >>= 1) bytes += __shfl_xor_sync(0xFFFFFFFFu, bytes, m);
            const bool rng_bad = __any_sync(0xFFFFFFFFu, lane < static_cast<int>(nr) &&
                                                             (hi < lo || hi - lo > static_cast<uint64_t>(kFmsChunk) ||
                                                              hi > dn));
            if (rng_bad || n_tot == 0 || n_tot > static_cast<uint32_t>(kFmsChunk) ||
                t_tot > static_cast<uint32_t>(kFmsTagBytes)) {
                // cannot happen for runs in start order (a chunk holds 1 ..
                // kFmsChunk records): the copies are not issued, and the sweep
                // reports a time-out -- or, when the runs were given, records
                // out of start order (a given run that is not in order can
                // split unevenly)
                if (lane == 0) {
                    const uint32_t why = given ? ST_UNSORTED : ST_TIMEOUT;
                    if (!given) atomicOr(gstatus, ST_TIMEOUT);
                    atomicOr(segs[ctl->list[k]].status, why);
                    MT.valid = 0;
                    mbar_arrive(&sh.full[s]);
                }
                break;
            }
            if (lane < static_cast<int>(nr)) {
                MT.roff[lane] = ro;
                MT.tpos[lane] = to + static_cast<uint32_t>(A & 15u);
                MT.direct[lane] = direct;
                MT.lo[lane] = lo;
            }
            if (lane < kSegCopyWords) reinterpret_cast<int64_t*>(&MT.sd)[lane] = sdw;
            if (lane == 0) {
                MT.roff[nr] = n_tot;
                MT.g = g;
                MT.sc = sc;
                MT.k = k;
                MT.c = c;
                MT.nr = nr;
                MT.n = n_tot;
                MT.valid = 1;
                MT.first = FIX ? 0u : (first ? 1u : 0u);
                MT.last = FIX ? 0u : (g + 1 == g_end ? 1u : 0u);
                MT.seg_first = FIX ? 0u : (sc == scb ? 1u : 0u);
                MT.given = given;
                MT.LK = LK;
                MT.LM = LM;
                MT.TK = TK;
                MT.TM = TM;
            }
            __syncwarp();
            // lane 0's arrive releases the meta fields written by every lane
            if (lane == 0) mbar_arrive_expect_tx(&sh.full[s], bytes);
            __syncwarp();
            if (lane < static_cast<int>(nr) && len) {
                tma_load_1d(&S.rows[ro], dse + 2 * lo, len * 16u, &sh.full[s]);
                if (tb) tma_load_1d(&S.tags[to], reinterpret_cast<const void*>(tlo), tb, &sh.full[s]);
            }
            first = false;
            if (!FIX) ++g;
        }
        return;
    }

    // -------------------------------------------------------- consumers
    const int ct = threadIdx.x - 32, cw = ct >> 5;
    for (uint32_t it = 0;; ++it) {
        const int s = static_cast<int>(it % kFmsStages);
        FmsStage& S = sh.st[s];
        // every stage completes one phase of full[s]: filled by bulk copies, or
        // (no more chunks) by a plain arrive
        const bool okw = mbar_wait_bounded(&sh.full[s], (it / kFmsStages) & 1u, wait_limit);
        if (!okw) atomicAdd(&sh.tmo, 1u);
        cbar();
        if (sh.tmo) {   // a wait ran out somewhere in the CTA: every consumer stops
            if (ct == 0) atomicOr(gstatus, ST_TIMEOUT);
            break;
        }
        const ChunkMeta& M = sh.meta[it & 1];
        if (!M.valid) break;   // no more chunks
        const uint32_t n = M.n, nr = M.nr;
        const SegCopy& d = M.sd;
        const int R = static_cast<int>(d.R);
        if (ct < 2 * R) sh.win[ct] = d.win[ct];
        if (ct == 0) sh.bad = 0;
        const uint32_t E = items_for(n);
        // the carry into this chunk
        int64_t LK, LM;
        if (FIX) {
            LK = M.LK;
            LM = M.LM;
        } else if (M.first) {
            LK = M.seg_first ? d.cin[0] : NEG_INF;
            LM = M.seg_first ? d.cin[1] : NEG_INF;
        } else {
            LK = sh.LK;
            LM = sh.LM;
        }
        const int64_t scK0 = M.first ? NEG_INF : sh.scK, scM0 = M.first ? NEG_INF : sh.scM;
        // tags the bulk copy could not fetch (past the last 16-byte boundary of the array)
        bool wrote = false;
        for (uint32_t q = 0; q < nr; ++q) {
            const uint32_t rl = M.roff[q + 1] - M.roff[q];
            for (uint32_t j = M.direct[q] + ct; j < rl; j += kFmsCT) {
                S.tags[M.tpos[q] + j] = d.tag[M.lo[q] + j];
                wrote = true;
            }
        }
        // the stage's next bulk copies must land after these writes
        if (wrote) fence_proxy_async_smem();
        cbar();

        // ---- aggregate, validation and span of the chunk's records.  Each
        // run's range is in start order, so the smallest and largest starts
        // are at the ranges' ends; the largest ends are taken relative to the
        // smallest start in 32 bits (hardware warp reductions) when the span
        // allows, else in 64 bits.
        int64_t s0 = INT64_MAX, mxS = NEG_INF;
        for (uint32_t q = 0; q < nr; ++q) {
            if (M.roff[q + 1] > M.roff[q]) {
                s0 = min64(s0, S.rows[M.roff[q]].x);
                mxS = max64(mxS, S.rows[M.roff[q + 1] - 1].x);
            }
        }
        uint32_t bK = 0, bM = 0, hib = 0, bad = 0;
        const bool given = M.given != 0;
        for (uint32_t q = 0; q < nr; ++q) {
            // this thread's records of run q: the staging indexes i == ct
            // (mod kFmsCT) in [a, b)
            const uint32_t a = M.roff[q], b = M.roff[q + 1];
            const uint32_t tp = M.tpos[q] - a;
            const uint32_t i0 = a + ((static_cast<uint32_t>(ct) + kFmsCT - a % kFmsCT) % kFmsCT);
            for (uint32_t i = i0; i < b; i += kFmsCT) {
                const longlong2 v = S.rows[i];
                const uint32_t tg = S.tags[tp + i];
                sh.tagc[i] = static_cast<uint8_t>(tg);
                bad |= (v.y < v.x) ? ST_BAD_END : 0u;
                bad |= (tg >= 160u) ? ST_BAD_KIND : 0u;
                const int64_t de = v.y - s0;
                hib |= static_cast<uint32_t>(static_cast<uint64_t>(de) >> 32);
                const uint32_t r = static_cast<uint32_t>(de);
                sh.key[0][i] = static_cast<uint32_t>(v.x - s0);   // used only when the span allows
                sh.end32[i] = r;
                // runs from the caller: each must be in start order (runs found
                // by the min/max pass or the sweep's run log are)
                if (given && i > a && S.rows[i - 1].x > v.x) bad |= ST_UNSORTED;
                if (tg < 32u) bK = umax(bK, r); else bM = umax(bM, r);
            }
        }
        if (given && ct < static_cast<int>(nr) && M.roff[ct + 1] > M.roff[ct] &&
            M.lo[ct] > ctl->runs[static_cast<uint64_t>(M.k) * (kMaxRuns + 1) + ct] &&
            d.se[2 * (M.lo[ct] - 1)] > S.rows[M.roff[ct]].x)
            bad |= ST_UNSORTED;   // a given run out of order across the chunk's boundary
        bK = __reduce_max_sync(0xFFFFFFFFu, bK);
        bM = __reduce_max_sync(0xFFFFFFFFu, bM);
        hib = __reduce_or_sync(0xFFFFFFFFu, hib);
        bad = __reduce_or_sync(0xFFFFFFFFu, bad);
        if ((ct & 31) == 0) {
            sh.red32[cw][0] = bK;
            sh.red32[cw][1] = bM;
            sh.red32[cw][2] = hib;
            sh.red32[cw][3] = bad;
        }
        cbar();
        bK = bM = hib = bad = 0;
#pragma unroll
        for (int q = 0; q < kFmsConsumers; ++q) {
            bK = umax(bK, sh.red32[q][0]);
            bM = umax(bM, sh.red32[q][1]);
            hib |= sh.red32[q][2];
            bad |= sh.red32[q][3];
        }
        // starts within 2^32 - 2 ns of s0: a 32-bit key never equals the
        // merge's end-of-run sentinel 0xFFFFFFFF
        const bool span32 = hib == 0 && static_cast<uint64_t>(mxS - s0) < 0xFFFFFFFFull;
        // 0 stands for "no record" (an end equal to s0 reads as none: it cannot
        // reach past any later start, so carries and sums are unchanged)
        int64_t aK = bK ? s0 + bK : NEG_INF, aM = bM ? s0 + bM : NEG_INF;
        if (!span32) {   // a chunk spanning 2^32 ns or more: the largest ends in 64 bits
            aK = aM = NEG_INF;
            uint32_t q = 0;
            for (uint32_t i = ct; i < n; i += kFmsCT) {
                while (i >= M.roff[q + 1]) ++q;
                const int64_t e = S.rows[i].y;
                if (sh.tagc[i] < 32u) aK = max64(aK, e); else aM = max64(aM, e);
            }
            aK = warp_max64(aK);
            aM = warp_max64(aM);
            cbar();   // every red32 read above is done before red64 is reused
            if ((ct & 31) == 0) {
                sh.red64[cw][0] = aK;
                sh.red64[cw][1] = aM;
            }
            cbar();
            aK = aM = NEG_INF;
#pragma unroll
            for (int q = 0; q < kFmsConsumers; ++q) {
                aK = max64(aK, sh.red64[q][0]);
                aM = max64(aM, sh.red64[q][1]);
            }
        }
        if (FIX) bad = 0;   // reported by the main pass
        // APPEND: the slice starts no earlier than the device's last ingested record
        if (!FIX && M.c == 0 && s0 < d.cin[2]) bad |= ST_UNSORTED;
        if (!FIX && ct == 0) {
            FmsChunk& fc = ctl->fms_chunk[M.g];
            fc.aggK = aK;
            fc.aggM = aM;
            fc.LK = LK;
            fc.LM = LM;
            fc.s0 = s0;
            sh.LK = max64(LK, aK);
            sh.LM = max64(LM, aM);
            sh.scK = max64(scK0, aK);
            sh.scM = max64(scM0, aM);
            if (M.last) {
                ctl->fms_sc_agg[2 * M.sc] = max64(scK0, aK);
                ctl->fms_sc_agg[2 * M.sc + 1] = max64(scM0, aM);
            }
        }

        // ---- merged order and the sweep (the barrier after the aggregate's
        // reduction above also published the compact arrays)
        const int64_t spanHi = max64(aK, aM);
        const int64_t hiK = FIX ? max64(M.TK, LK) : LK, hiM = FIX ? max64(M.TM, LM) : LM;
        const bool fast = span32 && (hiK <= s0 || ((hiK - s0) >> 32) == 0) && (hiM <= s0 || ((hiM - s0) >> 32) == 0);
        // the 32-bit path reads only the compact arrays from here on: the
        // stage goes back to the producer now (every read of it ended at the
        // barrier after the aggregate)
        const bool early = fast;
        if (early && ct == 0) mbar_arrive(&sh.empty[s]);
        const uint16_t* perm = nullptr;
        if (fast) {
            const uint32_t p0 = static_cast<uint32_t>(ct) * E;
            const int cnt = p0 < n ? static_cast<int>(min(E, n - p0)) : 0;
            uint32_t sr[kFmsItems], er[kFmsItems], tg[kFmsItems];
            merge32(sh, M, ct, E, cnt, sr, er, tg);
            uint32_t bK = 0, bM = 0;
            bool okE = true, okS = true, okK = true;
            dev_pass1<kFmsItems, false>(sr, er, tg, cnt, bK, bM, okE, okS, okK);
            // order self-check of the merge, inside the thread and across lanes
            uint32_t last = 0;
#pragma unroll
            for (int q = 0; q < kFmsItems; ++q)
                if (q < cnt) last = sr[q];
            const uint32_t prev_last = __shfl_up_sync(0xFFFFFFFFu, last, 1);
            uint32_t mybad = okS ? 0u : ST_UNSORTED;
            if (cnt > 0 && (ct & 31) > 0 && prev_last > sr[0]) mybad |= ST_UNSORTED;
            mybad = __reduce_or_sync(0xFFFFFFFFu, mybad);
            if ((ct & 31) == 0 && mybad) atomicOr(&sh.bad, mybad);
            if (FIX) {
                sweep32(sh, s0, spanHi, ct, cnt, R, sr, er, tg, bK, bM, M.TK, M.TM, d.sums, 1);
                sweep32(sh, s0, spanHi, ct, cnt, R, sr, er, tg, bK, bM, LK, LM, d.sums, -1);
            } else {
                sweep32(sh, s0, spanHi, ct, cnt, R, sr, er, tg, bK, bM, LK, LM, d.sums, 1);
            }
        } else {
            perm = sh.ix[merge_rounds(sh, S, M, ct, E)];
            if (FIX) {
                sweep64(sh, S, M, perm, ct, E, R, M.TK, M.TM, d.sums, 1);
                sweep64(sh, S, M, perm, ct, E, R, LK, LM, d.sums, -1);
            } else {
                sweep64(sh, S, M, perm, ct, E, R, LK, LM, d.sums, 1);
            }
            // order self-check of the merge
            const uint32_t p0 = static_cast<uint32_t>(ct) * E;
            uint32_t mybad = 0;
            for (uint32_t p = max(p0, 1u); p < min(n, p0 + E); ++p)
                if (S.rows[perm[p - 1]].x > S.rows[perm[p]].x) mybad = ST_UNSORTED;
            if (mybad) atomicOr(&sh.bad, mybad);
        }
        cbar();
        if (ct == 0) {
            const uint32_t bits = bad | sh.bad;
            if (bits) {
                atomicOr(d.status, bits);
                atomicOr(&seg_flags[d.seg], bits);
            }
            if (!FIX) {
                atomic_max64(&d.cout[0], aK);
                atomic_max64(&d.cout[1], aM);
                atomic_max64(&d.cout[2], mxS);
            }
            if (!early) mbar_arrive(&sh.empty[s]);
        }
    }
}

// ------------------------------------------------------------------ fix-up
// One warp per fused segment, 32 super-chunks at a time: the true carry of
// each super-chunk (the largest ends before it in its segment, earlier
// ingests included) by a max-scan over the super-chunks' aggregates, against
// the carries its chunks were swept with; the leading chunks whose carry was
// smaller, and whose records start below the true carry, become fix-up jobs.
__global__ void __launch_bounds__(256) fms_fix_plan_kernel(const SegDesc* __restrict__ segs, SortCtl* ctl) {
    const int lane = threadIdx.x & 31;
    const uint32_t nflag = ctl->nflag;
    const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint32_t nw = gridDim.x * (blockDim.x >> 5);
    for (uint32_t k = gw; k < nflag; k += nw) {
        const uint64_t sb = ctl->fms_sc_base[k], se = ctl->fms_sc_base[k + 1];
        if (sb == se) continue;
        const SegDesc& d = segs[ctl->list[k]];
        int64_t CK = d.carry_in[0], CM = d.carry_in[1];   // everything before the current group
        for (uint64_t j = sb; j < se; j += 32) {
            const uint64_t sc = j + lane;
            int64_t aK = NEG_INF, aM = NEG_INF;
            if (sc < se) {
                aK = ctl->fms_sc_agg[2 * sc];
                aM = ctl->fms_sc_agg[2 * sc + 1];
            }
            int64_t iK = aK, iM = aM;
            warp_incl_max2(iK, iM, lane);
            int64_t TK = shfl_up64(iK, 1), TM = shfl_up64(iM, 1);
            if (lane == 0) TK = TM = NEG_INF;
            TK = max64(TK, CK);
            TM = max64(TM, CM);
            CK = max64(CK, shfl64(iK, 31));
            CM = max64(CM, shfl64(iM, 31));
            if (sc < se && sc > sb) {   // the first super-chunk was swept with the true carry
                const uint64_t g0 = ctl->fms_chunk_base[k] + (sc - sb) * kFmsSuper;
                const uint64_t g1 = min(g0 + static_cast<uint64_t>(kFmsSuper), ctl->fms_chunk_base[k + 1]);
                for (uint64_t g = g0; g < g1; ++g) {
                    const FmsChunk fc = ctl->fms_chunk[g];
                    // the carry matters only where it passes the chunk's carry and a start
                    if (!(TK > fc.LK || TM > fc.LM) || max64(TK, TM) <= fc.s0) break;
                    const uint32_t q = atomicAdd(&ctl->fms_nfix, 1u);
                    ctl->fms_fix[q] = FmsFix{g, max64(TK, fc.LK), max64(TM, fc.LM)};
                }
            }
        }
    }
}

}  // namespace

static int g_fms_grid = 0;

cudaError_t fms_prepare(int num_sms) {
    if (g_fms_grid) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fms_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sizeof(FmsShared)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fms_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(sizeof(FmsShared)));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fms_kernel<false>, kFmsThreads, sizeof(FmsShared));
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    g_fms_grid = per_sm * num_sms;
    return cudaSuccess;
}

cudaError_t launch_fms(const SegDesc* segs, SortCtl* ctl, uint32_t* seg_flags, uint32_t* gstatus, int64_t wait_limit,
                       int grid_samples, cudaStream_t stream) {
    if (!g_fms_grid) return cudaErrorInvalidConfiguration;
    fms_plan_kernel<<<1, 1024, 0, stream>>>(ctl);
    fms_sample_kernel<<<grid_samples, 256, 0, stream>>>(segs, ctl);
    fms_split_kernel<<<grid_samples, 256, 0, stream>>>(segs, ctl);
    fms_kernel<false><<<g_fms_grid, kFmsThreads, sizeof(FmsShared), stream>>>(segs, ctl, seg_flags, gstatus,
                                                                               wait_limit);
    fms_fix_plan_kernel<<<grid_samples, 256, 0, stream>>>(segs, ctl);
    fms_kernel<true><<<g_fms_grid, kFmsThreads, sizeof(FmsShared), stream>>>(segs, ctl, seg_flags, gstatus,
                                                                              wait_limit);
    return cudaGetLastError();
}

uint64_t fms_max_samples(uint64_t n) { return n / kFmsMinStep + kMaxRuns + 1; }
uint64_t fms_max_chunks(uint64_t n) { return (4 * n + kFmsChunk - 1) / kFmsChunk + 2; }
uint64_t fms_max_super(uint64_t n) { return fms_max_chunks(n) / kFmsSuper + 1; }

}  // namespace talp
