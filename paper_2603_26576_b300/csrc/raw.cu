// Raw activity-record adapter: device records as an activity API delivers
// them (Sec. 4.2: buffers of records handed over when full or flushed,
// records of all of a process's devices and streams interleaved in
// completion order) are laid out as the per-device lanes the reduction
// reads.
//
// Per rank, every record goes to bucket (local device, stream); a stable
// counting scatter (per-tile bucket counts, a per-rank scan over tiles and
// buckets, then ranks inside the tile from warp matches and per-warp
// counters) writes each device's lane as its streams one after another,
// each stream in delivery order.  A stream executes in order, so each
// stream is already in start order and the lane is a few sorted runs,
// which the sort stage merges.
//
// Hold-back (buffers streamed over several calls): a later buffer may still
// bring a record that starts before records already delivered on other
// streams of its device.  A stream's later records start no earlier than
// its last delivered start, so the records of a device that start at or
// before W = min over its declared streams of their last delivered start
// are final and fold now; the rest are held back and delivered again,
// ahead of the next buffer's records, or folded by a flush.
#include "kernels.h"

namespace talp {

namespace {

constexpr int kRawThreads = 256;
constexpr int kRawItems = 8;
constexpr int kRawTile = kRawThreads * kRawItems;   // records per tile
constexpr int kBuckets = kRawBuckets;               // (local device, stream)

__device__ __forceinline__ uint32_t bucket_of(uint8_t dev, uint8_t tag) { return dev * 32u + (tag & 31u); }

// per tile: how many of its records fall in each bucket
__global__ void __launch_bounds__(kRawThreads) raw_hist_kernel(const RawTile* __restrict__ tiles, uint32_t n_tiles,
                                                               const RawRank* __restrict__ ranks,
                                                               uint32_t* __restrict__ hist, uint32_t* __restrict__ status) {
    __shared__ uint32_t h[kBuckets];
    for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const RawTile tl = tiles[t];
        const uint32_t D = ranks[tl.rank].D;
        for (int b = threadIdx.x; b < kBuckets; b += kRawThreads) h[b] = 0;
        __syncthreads();
        // all the tile's device and tag bytes loaded first, then one
        // shared-memory add per record
        uint8_t dv[kRawItems], tv[kRawItems];
#pragma unroll
        for (int r = 0; r < kRawItems; ++r) {
            const uint32_t q = r * kRawThreads + threadIdx.x;
            dv[r] = q < tl.n ? tl.dev[q] : 0xFF;
            tv[r] = q < tl.n ? tl.tag[q] : 0;
        }
#pragma unroll
        for (int r = 0; r < kRawItems; ++r) {
            const uint32_t q = r * kRawThreads + threadIdx.x;
            if (q < tl.n) {
                if (dv[r] < D) atomicAdd(&h[bucket_of(dv[r], tv[r])], 1u);
                else atomicOr(status, 1u);
            }
        }
        __syncthreads();
        for (int b = threadIdx.x; b < kBuckets; b += kRawThreads) hist[static_cast<uint64_t>(t) * kBuckets + b] = h[b];
        __syncthreads();
    }
}

// per rank: output position of every (tile, bucket), each bucket's lane
// range and each device's count
// The runs of a device lane made of its streams one after another (each
// stream in start order): the boundaries between its non-empty streams.
// Written as a known-runs record (count r, then the r + 1 boundaries), or
// count 0 when the lane has fewer than 2 or more than kMaxRuns non-empty
// streams (the sort stage then finds the runs itself).  cnt(s): records of
// stream s in the lane.
template <typename F>
__device__ __forceinline__ void write_runs(uint64_t* rec, F cnt) {
    uint32_t r = 0;
    for (int s = 0; s < 32; ++s) r += cnt(s) ? 1u : 0u;
    if (r < 2 || r > static_cast<uint32_t>(kMaxRuns)) {
        rec[0] = 0;
        return;
    }
    rec[0] = r;
    uint64_t at = 0;
    uint32_t j = 0;
    rec[1] = 0;
    for (int s = 0; s < 32; ++s) {
        const uint64_t c = cnt(s);
        if (c) {
            at += c;
            rec[2 + j++] = at;
        }
    }
}

__global__ void __launch_bounds__(kBuckets) raw_scan_kernel(const RawRank* __restrict__ ranks, uint32_t n_ranks,
                                                            const uint32_t* __restrict__ hist, uint64_t* __restrict__ offs,
                                                            RawMove* __restrict__ moves, uint64_t* __restrict__ dev_count,
                                                            uint32_t* __restrict__ dev_streams,
                                                            uint64_t* __restrict__ dev_runs) {
    __shared__ uint64_t s_tot[kBuckets];
    const uint32_t b = threadIdx.x;
    for (uint32_t r = blockIdx.x; r < n_ranks; r += gridDim.x) {
        const RawRank rk = ranks[r];
        const uint32_t te = rk.tile0 + rk.ntile;
        uint64_t tot = 0;
        uint32_t t = rk.tile0;
        for (; t + 8 <= te; t += 8) {   // 8 independent loads in flight per thread
            uint32_t v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = hist[static_cast<uint64_t>(t + i) * kBuckets + b];
#pragma unroll
            for (int i = 0; i < 8; ++i) tot += v[i];
        }
        for (; t < te; ++t) tot += hist[static_cast<uint64_t>(t) * kBuckets + b];
        s_tot[b] = tot;
        __syncthreads();
        uint64_t base = 0;
        for (uint32_t q = 0; q < b; ++q) base += s_tot[q];
        uint64_t run = rk.out0 + base;
        if (moves) {
            RawMove mv;
            mv.src = run;
            mv.fold_dst = mv.hold_dst = 0;
            mv.nfold = static_cast<uint32_t>(tot);
            mv.nhold = 0;
            moves[static_cast<uint64_t>(r) * kBuckets + b] = mv;
        }
        t = rk.tile0;
        for (; t + 8 <= te; t += 8) {
            uint32_t v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = hist[static_cast<uint64_t>(t + i) * kBuckets + b];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                offs[static_cast<uint64_t>(t + i) * kBuckets + b] = run;
                run += v[i];
            }
        }
        for (; t < te; ++t) {
            offs[static_cast<uint64_t>(t) * kBuckets + b] = run;
            run += hist[static_cast<uint64_t>(t) * kBuckets + b];
        }
        if (b < rk.D) {
            uint64_t c = 0;
            uint32_t ns = 0;
            for (int s = 0; s < 32; ++s) {
                c += s_tot[b * 32 + s];
                ns += s_tot[b * 32 + s] ? 1u : 0u;
            }
            dev_count[rk.dev0 + b] = c;
            dev_streams[rk.dev0 + b] = ns;
            if (dev_runs)
                write_runs(dev_runs + static_cast<uint64_t>(rk.dev0 + b) * kRunsStride,
                           [&](int q) { return s_tot[b * 32 + q]; });
        }
        __syncthreads();
    }
}

// stable scatter: warp w ranks records [w * 256, (w + 1) * 256) of the tile
__global__ void __launch_bounds__(kRawThreads) raw_scatter_kernel(const RawTile* __restrict__ tiles, uint32_t n_tiles,
                                                                  const RawRank* __restrict__ ranks,
                                                                  const uint64_t* __restrict__ offs,
                                                                  int64_t* __restrict__ lse, uint8_t* __restrict__ ltag,
                                                                  uint32_t* __restrict__ status, int64_t wait_limit) {
    __shared__ uint32_t cnt[kRawThreads / 32][kBuckets];
    __shared__ uint64_t s_offs[kBuckets];   // the tile's lane offset of every bucket
    // the tile's 16-byte rows, brought in by one bulk copy while the tile is ranked
    __shared__ __align__(16) longlong2 rows[kRawTile];
    __shared__ __align__(8) uint64_t bar;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const RawTile tl = tiles[t];
        const uint32_t D = ranks[tl.rank].D;
        if (threadIdx.x == 0 && tl.n) {
            fence_proxy_async_smem();   // the previous tile's reads of `rows` come first
            mbar_arrive_expect_tx(&bar, tl.n * 16u);
            tma_load_1d(rows, tl.se, tl.n * 16u, &bar);
        }
        for (int q = threadIdx.x; q < (kRawThreads / 32) * kBuckets; q += kRawThreads) (&cnt[0][0])[q] = 0;
        for (int q = threadIdx.x; q < kBuckets; q += kRawThreads) s_offs[q] = offs[static_cast<uint64_t>(t) * kBuckets + q];
        __syncthreads();
        const uint32_t w0 = wid * (kRawTile / (kRawThreads / 32));
        uint32_t bk[kRawItems], rnk[kRawItems];
        bool ok[kRawItems];
        uint8_t tv[kRawItems];
#pragma unroll
        for (int r = 0; r < kRawItems; ++r) {   // the lane's device and tag bytes, loaded first
            const uint32_t q = w0 + r * 32 + lane;
            const uint8_t dv = q < tl.n ? tl.dev[q] : 0xFF;
            tv[r] = q < tl.n ? tl.tag[q] : 0;
            ok[r] = dv < D;
            bk[r] = ok[r] ? bucket_of(dv, tv[r]) : kBuckets + lane;   // unique when unused
        }
#pragma unroll
        for (int r = 0; r < kRawItems; ++r) {
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, bk[r]);
            const uint32_t below = __popc(peers & ((1u << lane) - 1u));
            uint32_t basec = 0;
            if (ok[r]) basec = cnt[wid][bk[r]];
            rnk[r] = basec + below;
            __syncwarp();
            if (ok[r] && below == 0) cnt[wid][bk[r]] = basec + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per bucket, exclusive prefix over the warps
        for (int b = threadIdx.x; b < kBuckets; b += kRawThreads) {
            uint32_t run = 0;
            for (int w = 0; w < kRawThreads / 32; ++w) {
                const uint32_t c = cnt[w][b];
                cnt[w][b] = run;
                run += c;
            }
        }
        __syncthreads();
        if (tl.n) {
            // bounded wait for the rows; past the limit the copy is still let
            // land (and the result reports the time-out) before anything reuses
            // the buffer, and a copy that never lands ends the CTA's work
            bool landed = mbar_wait_bounded(&bar, phase, wait_limit);
            if (!landed) {
                atomicOr(status, ST_TIMEOUT);
                landed = mbar_wait_bounded(&bar, phase, kDrainWaitCycles);
            }
            if (__syncthreads_or(!landed)) return;
            phase ^= 1u;
        }
#pragma unroll
        for (int r = 0; r < kRawItems; ++r) {
            if (ok[r]) {
                const uint32_t q = w0 + r * 32 + lane;
                const uint64_t o = s_offs[bk[r]] + cnt[wid][bk[r]] + rnk[r];
                *reinterpret_cast<longlong2*>(lse + 2 * o) = rows[q];
                ltag[o] = tv[r];
            }
        }
        __syncthreads();
    }
}

// Hold-back split, one CTA per rank, thread b = bucket (device b / 32 in
// warp b / 32, stream b % 32): the last delivered start of every stream,
// the device's watermark W (a warp min over its declared streams), the
// final prefix of each bucket (records starting at or before W, found by
// binary search: a bucket is in start order) and where both parts go.
__global__ void __launch_bounds__(kBuckets) raw_hold_kernel(const RawRank* __restrict__ ranks, uint32_t n_ranks,
                                                            const int64_t* __restrict__ lse,
                                                            RawMove* __restrict__ moves,
                                                            uint64_t* __restrict__ fold_count,
                                                            uint64_t* __restrict__ hold_count,
                                                            uint32_t* __restrict__ status,
                                                            uint64_t* __restrict__ dev_runs) {
    __shared__ uint32_t s_f[kBuckets], s_h[kBuckets];
    const uint32_t b = threadIdx.x;
    const uint32_t d = b >> 5, sidx = b & 31;
    for (uint32_t r = blockIdx.x; r < n_ranks; r += gridDim.x) {
        const RawRank rk = ranks[r];
        if (!rk.last_start) continue;   // uniform over the block
        RawMove mv = moves[static_cast<uint64_t>(r) * kBuckets + b];
        const uint32_t n = mv.nfold;    // the scan stored the bucket's count here
        const bool declared = d < rk.D && ((ranks[r].smask[d] >> sidx) & 1u);
        if (n && !declared) atomicOr(status, 2u);
        int64_t ls = INT64_MIN;
        if (d < rk.D) {
            ls = rk.fresh ? INT64_MIN : rk.last_start[b];
            if (n) ls = max64(ls, lse[2 * (mv.src + n - 1)]);
            rk.last_start[b] = ls;
        }
        int64_t W = declared ? ls : INT64_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) W = min64(W, shfl_xor64(W, o));
        uint32_t lo = 0, hi = n;   // records starting at or before W
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (lse[2 * (mv.src + mid)] <= W) lo = mid + 1;
            else hi = mid;
        }
        s_f[b] = lo;
        s_h[b] = n - lo;
        __syncthreads();
        uint32_t ef = 0, eh = 0, df = 0, rh = 0;
        for (uint32_t q = 0; q < kBuckets; ++q) {
            const uint32_t f = s_f[q], h = s_h[q];
            if (q < b) {
                ef += f;
                eh += h;
            }
            if ((q >> 5) == d) df += f;
            rh += h;
        }
        mv.fold_dst = ef;
        mv.hold_dst = eh;
        mv.nfold = lo;
        mv.nhold = n - lo;
        moves[static_cast<uint64_t>(r) * kBuckets + b] = mv;
        if (sidx == 0 && d < rk.D) {
            fold_count[rk.dev0 + d] = df;
            // the fold lane is each stream's final part, stream after stream
            if (dev_runs)
                write_runs(dev_runs + static_cast<uint64_t>(rk.dev0 + d) * kRunsStride,
                           [&](int q) { return static_cast<uint64_t>(s_f[d * 32 + q]); });
        }
        if (b == 0) hold_count[r] = rh;
        __syncthreads();
    }
}

// Moves the split lanes, tile by tile over each rank's lane records (tiles
// of the same sizes as its input's): a record at lane position p belongs to the last
// bucket starting at or before p; its final part goes to the fold lanes at
// the rank's fold base, the rest to the rank's held records.
__global__ void __launch_bounds__(kRawThreads) raw_move_kernel(const RawTile* __restrict__ tiles, uint32_t n_tiles,
                                                               const RawRank* __restrict__ ranks,
                                                               const RawMove* __restrict__ moves,
                                                               const uint64_t* __restrict__ fold_base,
                                                               const int64_t* __restrict__ lse,
                                                               const uint8_t* __restrict__ ltag,
                                                               int64_t* __restrict__ fse, uint8_t* __restrict__ ftag) {
    __shared__ RawMove s_mv[kBuckets];
    for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const uint32_t r = tiles[t].rank;
        const uint32_t n = tiles[t].n;
        const RawRank& rk = ranks[r];
        if (!rk.last_start) continue;   // uniform over the block
        const uint64_t p0 = tiles[t].lpos;
        const uint64_t fb = fold_base[r];
        int64_t* const hse = rk.hold_se;
        uint8_t* const htag = rk.hold_tag;
        uint8_t* const hdev = rk.hold_dev;
        for (int q = threadIdx.x; q < kBuckets; q += kRawThreads) s_mv[q] = moves[static_cast<uint64_t>(r) * kBuckets + q];
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < n; q += kRawThreads) {
            const uint64_t p = p0 + q;
            uint32_t lo = 0, hi = kBuckets - 1;   // last bucket with src <= p
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (s_mv[mid].src <= p) lo = mid;
                else hi = mid - 1;
            }
            const RawMove& mv = s_mv[lo];
            const uint32_t i = static_cast<uint32_t>(p - mv.src);
            const longlong2 v = *reinterpret_cast<const longlong2*>(lse + 2 * p);
            const uint8_t tg = ltag[p];
            if (i < mv.nfold) {
                const uint64_t o = fb + mv.fold_dst + i;
                *reinterpret_cast<longlong2*>(fse + 2 * o) = v;
                ftag[o] = tg;
            } else {
                const uint32_t o = mv.hold_dst + (i - mv.nfold);
                *reinterpret_cast<longlong2*>(hse + 2 * static_cast<uint64_t>(o)) = v;
                htag[o] = tg;
                hdev[o] = static_cast<uint8_t>(lo >> 5);
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_raw_count(const RawTile* tiles, uint32_t n_tiles, const RawRank* ranks, uint32_t n_ranks,
                             uint32_t* hist, uint64_t* offs, RawMove* moves, uint64_t* dev_count,
                             uint32_t* dev_streams, uint64_t* dev_runs, uint32_t* status, int grid,
                             cudaStream_t stream) {
    if (n_tiles) raw_hist_kernel<<<grid, kRawThreads, 0, stream>>>(tiles, n_tiles, ranks, hist, status);
    if (n_ranks)
        raw_scan_kernel<<<n_ranks < 65535u ? n_ranks : 65535u, kBuckets, 0, stream>>>(ranks, n_ranks, hist, offs,
                                                                                     moves, dev_count, dev_streams,
                                                                                     dev_runs);
    return cudaGetLastError();
}

cudaError_t launch_raw_scatter(const RawTile* tiles, uint32_t n_tiles, const RawRank* ranks, const uint64_t* offs,
                               int64_t* lse, uint8_t* ltag, uint32_t* status, int64_t wait_limit, int grid,
                               cudaStream_t stream) {
    if (n_tiles)
        raw_scatter_kernel<<<grid, kRawThreads, 0, stream>>>(tiles, n_tiles, ranks, offs, lse, ltag, status, wait_limit);
    return cudaGetLastError();
}

cudaError_t launch_raw_hold(const RawRank* ranks, uint32_t n_ranks, const int64_t* lse, RawMove* moves,
                            uint64_t* fold_count, uint64_t* hold_count, uint32_t* status, uint64_t* dev_runs,
                            cudaStream_t stream) {
    if (n_ranks)
        raw_hold_kernel<<<n_ranks < 65535u ? n_ranks : 65535u, kBuckets, 0, stream>>>(ranks, n_ranks, lse, moves,
                                                                                     fold_count, hold_count, status,
                                                                                     dev_runs);
    return cudaGetLastError();
}

cudaError_t launch_raw_move(const RawTile* tiles, uint32_t n_tiles, const RawRank* ranks, const RawMove* moves,
                            const uint64_t* fold_base, const int64_t* lse, const uint8_t* ltag, int64_t* fse,
                            uint8_t* ftag, int grid, cudaStream_t stream) {
    if (n_tiles)
        raw_move_kernel<<<grid, kRawThreads, 0, stream>>>(tiles, n_tiles, ranks, moves, fold_base, lse, ltag, fse, ftag);
    return cudaGetLastError();
}

int raw_tile_records() { return kRawTile; }

}  // namespace talp
