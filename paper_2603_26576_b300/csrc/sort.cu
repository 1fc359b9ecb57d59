// Sort stage: segmented LSD radix sort, by start, of the device segments the
// sweep found out of order, then a re-sweep of exactly those segments.
//
// The flattening of Sec. 4.2 needs every device's records in start order
// (order among equal starts is irrelevant: unions do not depend on it).  The
// sweep validates the order of every device segment as it streams it; only
// the flagged segments go through this stage, so input already in start
// order costs nothing here.
//
// Everything is device driven (no host round trip): a plan kernel compacts
// the flagged segments, a min/max kernel rebases each segment's keys to its
// smallest start, and each radix pass (8-bit digits) is three kernels:
// per-tile digit histograms, a per-segment scan of those histograms into
// output offsets, and a stable scatter (ranks from warp match + per-warp
// digit counters).  A segment needs only ceil(bits(max - min) / 8) passes;
// the kernels of a pass skip segments that are done.  The re-sweep then
// runs the ordinary sweep kernel over a segment table that points into the
// sorted copies.
//
// A flagged segment that is only a few sorted runs laid end to end (records
// grouped by stream, each stream in start order: the order per-stream
// activity buffers deliver) is not sorted here: a segment of at most
// kMaxRuns runs is merged and swept in one pass by the fused merge-sweep
// (fms.cu).  Where the start order descends comes from the first sweep's run
// log (it compares every pair of neighbouring records anyway), from the
// caller (a raw lane's streams), or else from the min/max kernel.
#include "kernels.h"

namespace talp {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;   // 2048 records

__device__ __forceinline__ int passes_for(int64_t mn, int64_t mx) {
    const uint64_t range = static_cast<uint64_t>(mx) - static_cast<uint64_t>(mn);
    const int bits = range ? 64 - __clzll(static_cast<long long>(range)) : 1;
    return (bits + 7) / 8;
}

// nruns of a flagged segment found already in start order (a presorted
// segment whose streams do not interleave): neither merged nor radix sorted,
// swept again from its own records
constexpr uint32_t kInOrder = 0xFFFFFFFFu;

// radix passes of flagged segment k (0 when it is merged and swept instead, or in order)
__device__ __forceinline__ int radix_passes(const SortCtl* ctl, uint32_t k) {
    return (ctl->fused[k] || ctl->nruns[k] == kInOrder) ? 0 : passes_for(ctl->mn[k], ctl->mx[k]);
}

// segment k of the flagged list owning tile t
__device__ __forceinline__ uint32_t seg_of_tile(const SortCtl* ctl, uint32_t t) {
    uint32_t lo = 0, hi = ctl->nflag;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (ctl->tile_base[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// In a grid-stride loop over tiles, the last tile before the first one of
// this CTA's stride class past segment k (the loop's increment lands there):
// skips the rest of a segment that has nothing to do in this launch.
__device__ __forceinline__ uint32_t skip_segment(const SortCtl* ctl, uint32_t k, uint32_t t) {
    const uint64_t end = ctl->tile_base[k + 1];
    const uint64_t steps = (end - t + gridDim.x - 1) / gridDim.x;
    return static_cast<uint32_t>(t + (steps - 1) * gridDim.x);
}

// ---------------------------------------------------------------- plan
__global__ void __launch_bounds__(1024) sort_plan_kernel(const SegDesc* __restrict__ segs, uint32_t n_segs,
                                                         const uint32_t* __restrict__ seg_flags, SortCtl* ctl) {
    __shared__ uint32_t s_cnt[32];
    __shared__ uint64_t s_rec[32], s_til[32];
    __shared__ uint32_t s_base, s_find;
    __shared__ uint64_t s_rbase, s_tbase;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        s_base = 0;
        s_find = 0;
        s_rbase = 0;
        s_tbase = 0;
    }
    __syncthreads();
    for (uint32_t c0 = 0; c0 < n_segs; c0 += blockDim.x) {
        const uint32_t s = c0 + tid;
        bool f = false;
        uint64_t n = 0;
        if (s < n_segs) {
            const SegDesc& d = segs[s];
            f = !d.is_host && (d.pad[0] & kSegSortable) &&
                ((seg_flags[s] & ST_UNSORTED) || (d.pad[0] & kSegPresort));
            n = f ? d.n : 0;
        }
        const uint64_t tiles = f ? (n + kSortTile - 1) / kSortTile : 0;
        // block-wide exclusive scans of (flag, n, tiles)
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, f);
        uint64_t wn = n, wt = tiles;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
            const uint64_t a = __shfl_up_sync(0xFFFFFFFFu, wn, dd);
            const uint64_t b = __shfl_up_sync(0xFFFFFFFFu, wt, dd);
            if (lane >= dd) {
                wn += a;
                wt += b;
            }
        }
        if (lane == 31) {
            s_cnt[wid] = __popc(bal);
            s_rec[wid] = wn;
            s_til[wid] = wt;
        }
        __syncthreads();
        uint32_t pc = 0;
        uint64_t pr = 0, pt = 0;
        for (int w = 0; w < wid; ++w) {
            pc += s_cnt[w];
            pr += s_rec[w];
            pt += s_til[w];
        }
        if (f) {
            const uint32_t k = s_base + pc + __popc(bal & ((1u << lane) - 1));
            ctl->list[k] = s;
            ctl->rec_base[k] = s_rbase + pr + wn - n;
            ctl->tile_base[k] = s_tbase + pt + wt - tiles;
            ctl->mn[k] = INT64_MAX;
            ctl->mx[k] = INT64_MIN;
            ctl->nruns[k] = 0;
            ctl->fused[k] = 0;
            ctl->given[k] = kRunsFound;
            const SegDesc& d = segs[s];
            // runs already known (a raw lane: its streams, one after another):
            // taken as they are, and the min/max pass leaves the segment alone
            const uint64_t* kr = ctl->known ? ctl->known[s] : nullptr;
            if (kr && kr[0] >= 2 && kr[0] <= static_cast<uint64_t>(kMaxRuns) && kr[1 + kr[0]] == d.n) {
                const uint32_t r = static_cast<uint32_t>(kr[0]);
                uint64_t* runs = ctl->runs + static_cast<uint64_t>(k) * (kMaxRuns + 1);
                for (uint32_t q = 0; q <= r; ++q) runs[q] = kr[1 + q];
                ctl->nruns[k] = r - 1;
                ctl->given[k] = kRunsKnown;
            } else if (ctl->seen_n && !(d.pad[0] & kSegPresort)) {
                // swept once already: its descents are in the run log, complete
                // when there are few enough (the merge plan puts them in order)
                const uint32_t c = ctl->seen_n[s];
                if (c >= 1 && c <= static_cast<uint32_t>(kMaxRuns - 1)) {
                    uint64_t* runs = ctl->runs + static_cast<uint64_t>(k) * (kMaxRuns + 1);
                    const uint64_t* sp = ctl->seen_pos + static_cast<uint64_t>(s) * kMaxRuns;
                    for (uint32_t q = 0; q < c; ++q) runs[1 + q] = sp[q];
                    ctl->nruns[k] = c;
                    ctl->given[k] = kRunsSeen;
                }
            }
            if (ctl->given[k] == kRunsFound) atomicAdd(&s_find, 1u);
            // the re-sweep recomputes this ingest's part of the segment: its
            // sums restart from their value before the ingest
            const int64_t* src = ctl->restore[s];
            for (int q = 0; q < 3 * d.R; ++q) d.sums[q] = src ? src[q] : 0;
            d.carry_out[0] = d.carry_in[0];
            d.carry_out[1] = d.carry_in[1];
            d.carry_out[2] = d.carry_in[2];
            atomicAnd(d.status, ~ST_UNSORTED);
        }
        __syncthreads();
        if (tid == blockDim.x - 1) {
            s_base += pc + __popc(bal);
            s_rbase += pr + wn;
            s_tbase += pt + wt;
        }
        __syncthreads();
    }
    if (tid == 0) {
        ctl->max_passes = 0;
        ctl->n_find = s_find;
        ctl->nflag = s_base;
        ctl->nrec = s_rbase;
        ctl->ntile = s_tbase;
        ctl->tile_base[s_base] = s_tbase;
    }
}

// ------------------------------------------------------------ min / max
__global__ void __launch_bounds__(kSortThreads) sort_minmax_kernel(const SegDesc* __restrict__ segs, SortCtl* ctl) {
    __shared__ int64_t s_mn[kSortThreads / 32], s_mx[kSortThreads / 32];
    if (ctl->n_find == 0) return;   // every flagged segment's runs are known already
    const uint32_t ntile = static_cast<uint32_t>(ctl->ntile);
    for (uint32_t t = blockIdx.x; t < ntile; t += gridDim.x) {
        const uint32_t k = seg_of_tile(ctl, t);
        if (ctl->given[k] != kRunsFound) {   // runs known already (block-uniform)
            t = skip_segment(ctl, k, t);
            continue;
        }
        const SegDesc& d = segs[ctl->list[k]];
        const uint64_t r0 = static_cast<uint64_t>(t - ctl->tile_base[k]) * kSortTile;
        int64_t mn = INT64_MAX, mx = INT64_MIN;
        uint64_t* runs = ctl->runs + static_cast<uint64_t>(k) * (kMaxRuns + 1);
        for (uint64_t j0 = r0; j0 < d.n && j0 < r0 + kSortTile; j0 += kSortThreads) {
            const uint64_t j = j0 + threadIdx.x;
            bool desc = false;
            if (j < d.n && j < r0 + kSortTile) {
                const int64_t s = d.se[2 * j];
                mn = min64(mn, s);
                mx = max64(mx, s);
                desc = j > 0 && s < d.se[2 * (j - 1)];
            }
            // positions where the start order descends (run starts); the
            // count goes on past kMaxRuns only to tell the segment is not a
            // few runs, so stop counting once it is far beyond
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, desc);
            uint32_t seen = 0;
            if (bal && (threadIdx.x & 31) == 0) seen = *static_cast<volatile uint32_t*>(&ctl->nruns[k]);
            seen = __shfl_sync(0xFFFFFFFFu, seen, 0);   // warp-uniform decision below
            if (bal && seen <= static_cast<uint32_t>(kMaxRuns)) {
                uint32_t base = 0;
                if ((threadIdx.x & 31) == 0) base = atomicAdd(&ctl->nruns[k], static_cast<uint32_t>(__popc(bal)));
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (desc) {
                    const uint32_t slot = base + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u));
                    if (slot < static_cast<uint32_t>(kMaxRuns)) runs[1 + slot] = j;
                }
            }
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
            mn = min64(mn, shfl_xor64(mn, m));
            mx = max64(mx, shfl_xor64(mx, m));
        }
        if ((threadIdx.x & 31) == 0) {
            s_mn[threadIdx.x >> 5] = mn;
            s_mx[threadIdx.x >> 5] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kSortThreads / 32; ++w) {
                mn = min64(mn, s_mn[w]);
                mx = max64(mx, s_mx[w]);
            }
            atomicMin(reinterpret_cast<long long*>(&ctl->mn[k]), static_cast<long long>(mn));
            atomicMax(reinterpret_cast<long long*>(&ctl->mx[k]), static_cast<long long>(mx));
        }
        __syncthreads();
    }
}

// source of pass p for flagged segment k: the original records, or the
// buffer written by the previous pass
__device__ __forceinline__ void pass_src(const SegDesc& d, const SortCtl* ctl, uint32_t k, int p,
                                         const int64_t*& se, const uint8_t*& tag) {
    if (p == 0) {
        se = d.se;
        tag = d.tag;
    } else {
        const int b = (p - 1) & 1;
        se = ctl->buf_se[b] + 2 * ctl->rec_base[k];
        tag = ctl->buf_tag[b] + ctl->rec_base[k];
    }
}

// ----------------------------------------------------------- histogram
__global__ void __launch_bounds__(kSortThreads) sort_hist_kernel(const SegDesc* __restrict__ segs, SortCtl* ctl,
                                                                 int p) {
    __shared__ uint32_t h[256];
    if (static_cast<uint32_t>(p) >= ctl->max_passes) return;
    const uint32_t ntile = static_cast<uint32_t>(ctl->ntile);
    for (uint32_t t = blockIdx.x; t < ntile; t += gridDim.x) {
        const uint32_t k = seg_of_tile(ctl, t);
        if (p >= radix_passes(ctl, k)) {   // block-uniform
            t = skip_segment(ctl, k, t);
            continue;
        }
        const SegDesc& d = segs[ctl->list[k]];
        const int64_t* se;
        const uint8_t* tag;
        pass_src(d, ctl, k, p, se, tag);
        h[threadIdx.x] = 0;
        __syncthreads();
        const uint64_t r0 = static_cast<uint64_t>(t - ctl->tile_base[k]) * kSortTile;
        const int64_t mn = ctl->mn[k];
        for (uint64_t j = r0 + threadIdx.x; j < d.n && j < r0 + kSortTile; j += kSortThreads) {
            const uint64_t key = static_cast<uint64_t>(se[2 * j]) - static_cast<uint64_t>(mn);
            atomicAdd(&h[(key >> (8 * p)) & 255u], 1u);
        }
        __syncthreads();
        ctl->hist[static_cast<uint64_t>(t) * 256 + threadIdx.x] = h[threadIdx.x];
        __syncthreads();
    }
}

// ----------------------------------------------------------------- scan
// hist[t][d] -> absolute output offset of tile t's first record of digit d
__global__ void __launch_bounds__(256) sort_scan_kernel(SortCtl* ctl, int p) {
    __shared__ uint32_t s_tot[256];
    if (static_cast<uint32_t>(p) >= ctl->max_passes) return;
    const uint32_t d = threadIdx.x;
    for (uint32_t k = blockIdx.x; k < ctl->nflag; k += gridDim.x) {
        if (p >= radix_passes(ctl, k)) continue;
        const uint64_t t0 = ctl->tile_base[k], t1 = ctl->tile_base[k + 1];
        uint64_t tot = 0;
        for (uint64_t t = t0; t < t1; ++t) tot += ctl->hist[t * 256 + d];
        s_tot[d] = static_cast<uint32_t>(tot);
        __syncthreads();
        uint64_t base = 0;
        for (uint32_t q = 0; q < d; ++q) base += s_tot[q];
        uint64_t run = ctl->rec_base[k] + base;
        for (uint64_t t = t0; t < t1; ++t) {
            const uint32_t v = ctl->hist[t * 256 + d];
            ctl->offs[t * 256 + d] = run;
            run += v;
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------- scatter
// Stable: the records of a tile are ranked in tile order; warp w owns the
// records [w*256, (w+1)*256) of the tile, in 8 rounds of 32.
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(const SegDesc* __restrict__ segs, SortCtl* ctl,
                                                                    int p) {
    __shared__ uint32_t cnt[kSortThreads / 32][256];
    if (static_cast<uint32_t>(p) >= ctl->max_passes) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t ntile = static_cast<uint32_t>(ctl->ntile);
    for (uint32_t t = blockIdx.x; t < ntile; t += gridDim.x) {
        const uint32_t k = seg_of_tile(ctl, t);
        if (p >= radix_passes(ctl, k)) {
            t = skip_segment(ctl, k, t);
            continue;
        }
        const SegDesc& d = segs[ctl->list[k]];
        const int64_t* se;
        const uint8_t* tag;
        pass_src(d, ctl, k, p, se, tag);
        int64_t* dse = ctl->buf_se[p & 1];
        uint8_t* dtag = ctl->buf_tag[p & 1];
        for (int q = threadIdx.x; q < (kSortThreads / 32) * 256; q += kSortThreads) (&cnt[0][0])[q] = 0;
        __syncthreads();
        const uint64_t r0 = static_cast<uint64_t>(t - ctl->tile_base[k]) * kSortTile + wid * 256;
        const int64_t mn = ctl->mn[k];
        longlong2 v[kSortItems];
        uint32_t tg[kSortItems], dg[kSortItems], rk[kSortItems];
        bool ok[kSortItems];
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const uint64_t j = r0 + r * 32 + lane;
            ok[r] = j < d.n && (j - (r0 - wid * 256)) < kSortTile;
            if (ok[r]) {
                v[r] = *reinterpret_cast<const longlong2*>(se + 2 * j);
                tg[r] = tag[j];
                dg[r] = ((static_cast<uint64_t>(v[r].x) - static_cast<uint64_t>(mn)) >> (8 * p)) & 255u;
            } else {
                dg[r] = 256u + lane;   // distinct from every digit and every other lane
            }
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, dg[r]);
            const uint32_t below = __popc(peers & ((1u << lane) - 1u));
            uint32_t basec = 0;
            if (ok[r]) basec = cnt[wid][dg[r]];
            rk[r] = basec + below;
            __syncwarp();
            if (ok[r] && below == 0) cnt[wid][dg[r]] = basec + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit, exclusive prefix over the warps
        {
            const int dd = threadIdx.x;
            uint32_t run = 0;
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const uint32_t c = cnt[w][dd];
                cnt[w][dd] = run;
                run += c;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            if (ok[r]) {
                const uint64_t o = ctl->offs[static_cast<uint64_t>(t) * 256 + dg[r]] + cnt[wid][dg[r]] + rk[r];
                *reinterpret_cast<longlong2*>(dse + 2 * o) = v[r];
                dtag[o] = static_cast<uint8_t>(tg[r]);
            }
        }
        __syncthreads();
    }
}


// --------------------------------------------------------------- merge plan
// One thread per flagged segment: a segment of 2 .. kMaxRuns sorted runs gets
// its run starts in order and is marked for the fused merge-sweep; any other
// goes to the radix sort (a presorted one found in order to neither).
__global__ void sort_merge_plan_kernel(const SegDesc* __restrict__ segs, SortCtl* ctl) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < ctl->nflag; k += gridDim.x * blockDim.x) {
        const uint32_t c = ctl->nruns[k];
        if (c == 0 && (segs[ctl->list[k]].pad[0] & kSegPresort)) {
            ctl->fused[k] = 0;
            ctl->nruns[k] = kInOrder;
            continue;
        }
        if (c == 0 || c + 1 > static_cast<uint32_t>(kMaxRuns)) {
            ctl->fused[k] = 0;
            atomicMax(&ctl->max_passes, static_cast<uint32_t>(passes_for(ctl->mn[k], ctl->mx[k])));
            continue;
        }
        uint64_t* runs = ctl->runs + static_cast<uint64_t>(k) * (kMaxRuns + 1);
        for (uint32_t i = 2; i <= c; ++i) {   // insertion sort of runs[1 .. c]
            const uint64_t v = runs[i];
            uint32_t q = i;
            while (q > 1 && runs[q - 1] > v) {
                runs[q] = runs[q - 1];
                --q;
            }
            runs[q] = v;
        }
        runs[0] = 0;
        runs[c + 1] = segs[ctl->list[k]].n;
        ctl->fused[k] = 1;
    }
}

// ------------------------------------------------------- re-sweep table
// Flagged segment k becomes segment k of a new table whose records are the
// sorted copy (or its own records, when found in order); fused segments
// (already swept) and slots nflag .. n_slots-1 are empty segments.
__global__ void __launch_bounds__(256) sort_resweep_plan_kernel(const SegDesc* __restrict__ segs, SortCtl* ctl,
                                                                SegDesc* out, uint64_t* out_start,
                                                                uint64_t* out_rend, uint32_t n_slots) {
    const uint32_t nflag = ctl->nflag;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k <= n_slots; k += gridDim.x * blockDim.x) {
        if (k == n_slots) {
            out_start[k] = ctl->nrec;
            continue;
        }
        if (k < nflag && !ctl->fused[k]) {
            SegDesc s = segs[ctl->list[k]];
            if (ctl->nruns[k] != kInOrder) {
                const int P = passes_for(ctl->mn[k], ctl->mx[k]);
                const int b = (P - 1) & 1;
                s.se = ctl->buf_se[b] + 2 * ctl->rec_base[k];
                s.tag = ctl->buf_tag[b] + ctl->rec_base[k];
                s.tag_limit = ctl->buf_tag_limit[b];
            }
            out[k] = s;
            out_start[k] = ctl->rec_base[k];
            out_rend[k] = ctl->rec_base[k] + s.n;
        } else {
            // no records; the table's starts stay non-decreasing (a fused
            // segment keeps its place, the unused slots sit at the end)
            SegDesc s = segs[0];
            s.n = 0;
            s.is_host = 1;
            s.R = 0;
            out[k] = s;
            const uint64_t at = k < nflag ? ctl->rec_base[k] : ctl->nrec;
            out_start[k] = at;
            out_rend[k] = at;
        }
    }
}

// Runs of a device whose records come grouped by stream (each stretch of
// consecutive records on one stream in start order, the caller's word): the
// positions where the stream id changes.  One block per segment reads its
// tags as aligned 16-byte blocks (thread t takes blocks t, t + 1024, ...: the
// loads coalesce) and compares every byte with the one before it (the block
// before comes from the previous lane, or for lane 0 from memory).  The
// boundaries go to a known-runs record (count r, then the r + 1 boundaries),
// or count 0 when there is a single stretch or more than kMaxRuns (the sort
// stage then finds the runs itself).  The merge-sweep checks every stretch
// for start order.  Reading whole aligned blocks may touch up to 15 bytes
// before and after the tags; each such block holds at least one tag byte, so
// it lies in mapped memory, and those bytes are ignored.
constexpr int kGroupThreads = 1024;
constexpr int kGroupCap = 64;   // boundaries kept (more: too many runs anyway)

__global__ void __launch_bounds__(kGroupThreads) group_runs_kernel(const SegDesc* __restrict__ segs, uint32_t n_segs,
                                                                   const uint64_t* const* __restrict__ known) {
    __shared__ uint32_t s_n;
    __shared__ uint64_t s_pos[kGroupCap];
    const uint32_t s = blockIdx.x;
    if (s >= n_segs) return;
    const SegDesc& d = segs[s];
    if (!(d.pad[0] & kSegGrouped)) return;   // uniform over the block
    uint64_t* rec = const_cast<uint64_t*>(known[s]);
    const uint64_t n = d.n;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    if (n > 1) {
        const uintptr_t A = reinterpret_cast<uintptr_t>(d.tag);
        const uintptr_t B0 = A & ~static_cast<uintptr_t>(15);
        const uint64_t nblk = (A + n - B0 + 15) / 16;
        // rounds of 1024 consecutive blocks; every thread takes part in every
        // round (the shuffles need the whole warp)
        for (uint64_t r0 = 0; r0 < nblk; r0 += kGroupThreads) {
            const uint64_t blk = r0 + threadIdx.x;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (blk < nblk) v = *reinterpret_cast<const uint4*>(B0 + 16 * blk);
            // the byte before the block: the last byte of the previous lane's
            // block, or (lane 0) read from memory
            uint32_t p = __shfl_up_sync(0xFFFFFFFFu, v.w >> 24, 1);
            if (lane == 0 && blk > 0 && blk < nblk) p = *reinterpret_cast<const uint8_t*>(B0 + 16 * blk - 1);
            const uint32_t m = 0x1F1F1F1Fu;
            const uint32_t d0 = (v.x ^ ((v.x << 8) | p)) & m;
            const uint32_t d1 = (v.y ^ ((v.y << 8) | (v.x >> 24))) & m;
            const uint32_t d2 = (v.z ^ ((v.z << 8) | (v.y >> 24))) & m;
            const uint32_t d3 = (v.w ^ ((v.w << 8) | (v.z >> 24))) & m;
            if ((d0 | d1 | d2 | d3) && blk < nblk) {   // rare: a stream changes somewhere in the block
                const uint32_t dw[4] = {d0, d1, d2, d3};
                for (int j = 0; j < 16; ++j) {
                    if ((dw[j >> 2] >> (8 * (j & 3))) & 0xFFu) {
                        // tag index of byte j; a boundary needs it and the byte
                        // before to be tags of the segment
                        const int64_t q = static_cast<int64_t>(B0 + 16 * blk + j) - static_cast<int64_t>(A);
                        if (q >= 1 && q < static_cast<int64_t>(n)) {
                            const uint32_t k = atomicAdd(&s_n, 1u);
                            if (k < static_cast<uint32_t>(kGroupCap)) s_pos[k] = static_cast<uint64_t>(q);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t c = s_n;   // boundaries: c + 1 runs
        if (c == 0 || c + 1 > static_cast<uint32_t>(kMaxRuns)) {
            rec[0] = 0;
        } else {
            // the boundaries in ascending order (at most kMaxRuns - 1 of them)
            for (uint32_t a = 1; a < c; ++a) {
                const uint64_t v = s_pos[a];
                uint32_t b = a;
                while (b > 0 && s_pos[b - 1] > v) {
                    s_pos[b] = s_pos[b - 1];
                    --b;
                }
                s_pos[b] = v;
            }
            rec[0] = c + 1;
            rec[1] = 0;
            for (uint32_t a = 0; a < c; ++a) rec[2 + a] = s_pos[a];
            rec[2 + c] = n;
        }
    }
}

}  // namespace

cudaError_t launch_sort_stage(const SegDesc* segs, uint32_t n_segs, uint32_t n_slots, uint32_t* seg_flags,
                              SortCtl* ctl, SegDesc* resweep_segs, uint64_t* resweep_start, uint64_t* resweep_rend,
                              int grid_tiles, int grid_segs, uint32_t* gstatus, int64_t wait_limit,
                              cudaStream_t stream) {
    if (n_slots == 0) return cudaSuccess;
    sort_plan_kernel<<<1, 1024, 0, stream>>>(segs, n_segs, seg_flags, ctl);
    sort_minmax_kernel<<<grid_tiles, kSortThreads, 0, stream>>>(segs, ctl);
    sort_merge_plan_kernel<<<grid_segs, 32, 0, stream>>>(segs, ctl);
    cudaError_t e = launch_fms(segs, ctl, seg_flags, gstatus, wait_limit, grid_tiles, stream);
    if (e != cudaSuccess) return e;
    for (int p = 0; p < 8; ++p) {
        sort_hist_kernel<<<grid_tiles, kSortThreads, 0, stream>>>(segs, ctl, p);
        sort_scan_kernel<<<grid_segs, 256, 0, stream>>>(ctl, p);
        sort_scatter_kernel<<<grid_tiles, kSortThreads, 0, stream>>>(segs, ctl, p);
    }
    const int g = static_cast<int>((n_slots + 1 + 255) / 256);
    sort_resweep_plan_kernel<<<g < 1024 ? g : 1024, 256, 0, stream>>>(segs, ctl, resweep_segs, resweep_start,
                                                                       resweep_rend, n_slots);
    return cudaGetLastError();
}

cudaError_t launch_group_runs(const SegDesc* segs, uint32_t n_segs, const uint64_t* const* known, cudaStream_t stream) {
    if (n_segs) group_runs_kernel<<<n_segs, kGroupThreads, 0, stream>>>(segs, n_segs, known);
    return cudaGetLastError();
}

int sort_tile_records() { return kSortTile; }

}  // namespace talp
