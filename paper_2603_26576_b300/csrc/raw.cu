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
#include "kernels.h"

namespace talp {

namespace {

constexpr int kRawThreads = 256;
constexpr int kRawItems = 8;
constexpr int kRawTile = kRawThreads * kRawItems;   // records per tile
constexpr int kBuckets = kRawMaxDevices * 32;       // (local device, stream)

__device__ __forceinline__ uint32_t bucket_of(uint8_t dev, uint8_t tag) { return dev * 32u + (tag & 31u); }

// per tile: how many of its records fall in each bucket
__global__ void __launch_bounds__(kRawThreads) raw_hist_kernel(const uint8_t* __restrict__ rdev,
                                                               const uint8_t* __restrict__ rtag,
                                                               const RawTile* __restrict__ tiles, uint32_t n_tiles,
                                                               const RawRank* __restrict__ ranks,
                                                               uint32_t* __restrict__ hist, uint32_t* __restrict__ status) {
    __shared__ uint32_t h[kBuckets];
    for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const RawTile tl = tiles[t];
        const uint32_t D = ranks[tl.rank].D;
        for (int b = threadIdx.x; b < kBuckets; b += kRawThreads) h[b] = 0;
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < tl.n; q += kRawThreads) {
            const uint8_t d = rdev[tl.rec0 + q];
            if (d >= D) {
                atomicOr(status, 1u);
                continue;
            }
            atomicAdd(&h[bucket_of(d, rtag[tl.rec0 + q])], 1u);
        }
        __syncthreads();
        for (int b = threadIdx.x; b < kBuckets; b += kRawThreads) hist[static_cast<uint64_t>(t) * kBuckets + b] = h[b];
        __syncthreads();
    }
}

// per rank: output position of every (tile, bucket) and each device's count
__global__ void __launch_bounds__(kBuckets) raw_scan_kernel(const RawRank* __restrict__ ranks, uint32_t n_ranks,
                                                            const uint32_t* __restrict__ hist, uint64_t* __restrict__ offs,
                                                            uint64_t* __restrict__ dev_count) {
    __shared__ uint64_t s_tot[kBuckets];
    const uint32_t b = threadIdx.x;
    for (uint32_t r = blockIdx.x; r < n_ranks; r += gridDim.x) {
        const RawRank rk = ranks[r];
        uint64_t tot = 0;
        for (uint32_t t = rk.tile0; t < rk.tile0 + rk.ntile; ++t) tot += hist[static_cast<uint64_t>(t) * kBuckets + b];
        s_tot[b] = tot;
        __syncthreads();
        uint64_t base = 0;
        for (uint32_t q = 0; q < b; ++q) base += s_tot[q];
        uint64_t run = rk.out0 + base;
        for (uint32_t t = rk.tile0; t < rk.tile0 + rk.ntile; ++t) {
            offs[static_cast<uint64_t>(t) * kBuckets + b] = run;
            run += hist[static_cast<uint64_t>(t) * kBuckets + b];
        }
        if (b < rk.D) {
            uint64_t c = 0;
            for (int s = 0; s < 32; ++s) c += s_tot[b * 32 + s];
            dev_count[rk.dev0 + b] = c;
        }
        __syncthreads();
    }
}

// stable scatter: warp w ranks records [w * 256, (w + 1) * 256) of the tile
__global__ void __launch_bounds__(kRawThreads) raw_scatter_kernel(const int64_t* __restrict__ rse,
                                                                  const uint8_t* __restrict__ rtag,
                                                                  const uint8_t* __restrict__ rdev,
                                                                  const RawTile* __restrict__ tiles, uint32_t n_tiles,
                                                                  const RawRank* __restrict__ ranks,
                                                                  const uint64_t* __restrict__ offs,
                                                                  int64_t* __restrict__ lse, uint8_t* __restrict__ ltag) {
    __shared__ uint32_t cnt[kRawThreads / 32][kBuckets];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const RawTile tl = tiles[t];
        const uint32_t D = ranks[tl.rank].D;
        for (int q = threadIdx.x; q < (kRawThreads / 32) * kBuckets; q += kRawThreads) (&cnt[0][0])[q] = 0;
        __syncthreads();
        const uint32_t w0 = wid * (kRawTile / (kRawThreads / 32));
        uint32_t bk[kRawItems], rnk[kRawItems];
        bool ok[kRawItems];
#pragma unroll
        for (int r = 0; r < kRawItems; ++r) {
            const uint32_t q = w0 + r * 32 + lane;
            ok[r] = q < tl.n && rdev[tl.rec0 + q] < D;
            bk[r] = ok[r] ? bucket_of(rdev[tl.rec0 + q], rtag[tl.rec0 + q]) : kBuckets + lane;   // unique when unused
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
#pragma unroll
        for (int r = 0; r < kRawItems; ++r) {
            if (ok[r]) {
                const uint32_t q = w0 + r * 32 + lane;
                const uint64_t o = offs[static_cast<uint64_t>(t) * kBuckets + bk[r]] + cnt[wid][bk[r]] + rnk[r];
                *reinterpret_cast<longlong2*>(lse + 2 * o) =
                    *reinterpret_cast<const longlong2*>(rse + 2 * (tl.rec0 + q));
                ltag[o] = rtag[tl.rec0 + q];
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_raw_count(const uint8_t* rdev, const uint8_t* rtag, const RawTile* tiles, uint32_t n_tiles,
                             const RawRank* ranks, uint32_t n_ranks, uint32_t* hist, uint64_t* offs,
                             uint64_t* dev_count, uint32_t* status, int grid, cudaStream_t stream) {
    if (n_tiles) raw_hist_kernel<<<grid, kRawThreads, 0, stream>>>(rdev, rtag, tiles, n_tiles, ranks, hist, status);
    if (n_ranks) raw_scan_kernel<<<n_ranks < 65535u ? n_ranks : 65535u, kBuckets, 0, stream>>>(ranks, n_ranks, hist,
                                                                                              offs, dev_count);
    return cudaGetLastError();
}

cudaError_t launch_raw_scatter(const int64_t* rse, const uint8_t* rtag, const uint8_t* rdev, const RawTile* tiles,
                               uint32_t n_tiles, const RawRank* ranks, const uint64_t* offs, int64_t* lse,
                               uint8_t* ltag, int grid, cudaStream_t stream) {
    if (n_tiles)
        raw_scatter_kernel<<<grid, kRawThreads, 0, stream>>>(rse, rtag, rdev, tiles, n_tiles, ranks, offs, lse, ltag);
    return cudaGetLastError();
}

int raw_tile_records() { return kRawTile; }

}  // namespace talp
