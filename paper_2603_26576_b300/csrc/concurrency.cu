// Concurrency profile of every device (the per-stream occupancy the paper
// leaves to future work, Sec. 4.1): for device g and one region window
// [a, b), with c(t) the number of g's records active at time t (records
// clipped to the window),
//   level[g][0][k-1] = |{t : c(t) >= k}|, k = 1 .. kConcLevels,
//   level[g][1][k-1] = the same over kernel records.
// Level 1 is the busy union B (resp. the kernel union D_K).
//
// With the records in start order, between the starts s_i and s_{i+1} of
// consecutive records exactly the records j <= i with e_j > t are active,
// so c(t) >= k there iff t < E_k(i), the k-th largest end among records
// j <= i: the time with c >= k in [s_i, s_{i+1}) is
//   max(0, min(s_{i+1}, E_k(i)) - s_i).
// A device's record list is cut into chunks; the top-K ends of each chunk
// are merged into every later chunk's entering state by a per-device scan,
// and each chunk then walks its records with a warp-wide scan of top-K
// lists per tile.  Top-K merges are bitonic (elementwise max against the
// reversed list, then a bitonic half-cleaner cascade).
#include "kernels.h"

namespace talp {

namespace {

constexpr int K = kConcLevels;
constexpr int kItems = 8;
constexpr int kTile = 32 * kItems;
constexpr int kWarps = 8;

// sorted-descending list of the K largest ends seen (INT64_MIN: none)
struct TopK {
    int64_t v[K];
};

__device__ __forceinline__ void cas_desc(int64_t& x, int64_t& y) {
    const int64_t hi = x > y ? x : y, lo = x > y ? y : x;
    x = hi;
    y = lo;
}

// top-K of the union of two sorted-descending lists (result sorted)
__device__ __forceinline__ void merge_top(TopK& x, const TopK& y) {
#pragma unroll
    for (int i = 0; i < K; ++i) x.v[i] = max64(x.v[i], y.v[K - 1 - i]);   // bitonic
#pragma unroll
    for (int w = K / 2; w > 0; w >>= 1) {
#pragma unroll
        for (int i = 0; i < K; ++i)
            if ((i & w) == 0) cas_desc(x.v[i], x.v[i + w]);
    }
}

__device__ __forceinline__ void insert_top(TopK& x, int64_t e) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int64_t hi = x.v[i] > e ? x.v[i] : e;
        e = x.v[i] > e ? e : x.v[i];
        x.v[i] = hi;
    }
}

__device__ __forceinline__ void clear_top(TopK& x) {
#pragma unroll
    for (int i = 0; i < K; ++i) x.v[i] = INT64_MIN;
}

__device__ __forceinline__ TopK shfl_top(const TopK& x, int src) {
    TopK y;
#pragma unroll
    for (int i = 0; i < K; ++i) y.v[i] = shfl64(x.v[i], src);
    return y;
}

__device__ __forceinline__ TopK shfl_up_top(const TopK& x, int d) {
    TopK y;
#pragma unroll
    for (int i = 0; i < K; ++i) y.v[i] = static_cast<int64_t>(__shfl_up_sync(0xFFFFFFFFu, static_cast<long long>(x.v[i]), d));
    return y;
}

// warp-inclusive scan of top-K lists over lanes
__device__ __forceinline__ void scan_top(TopK& x, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const TopK y = shfl_up_top(x, d);
        if (lane >= d) merge_top(x, y);
    }
}

// One tile of a chunk staged in shared memory: rows of 16 bytes and tags.
struct Stage {
    longlong2 se[kTile];
    uint8_t tag[kTile];
};

// Load the records [r0, r0 + n) of the record array into the warp's stage
// (n <= kTile), clipped to the window.
__device__ __forceinline__ void stage_tile(Stage& st, const int64_t* __restrict__ se, const uint8_t* __restrict__ tag,
                                           uint64_t r0, int n, int lane) {
    for (int q = lane; q < n; q += 32) {
        st.se[q] = *reinterpret_cast<const longlong2*>(se + 2 * (r0 + q));
        st.tag[q] = tag[r0 + q];
    }
    __syncwarp();
}

// ------------------------------------------------------------- chunk top-K
__global__ void __launch_bounds__(kWarps * 32) conc_chunk_top(const int64_t* __restrict__ se,
                                                             const uint8_t* __restrict__ tag,
                                                             const ConcDev* __restrict__ devs,
                                                             const ConcChunk* __restrict__ chunks, uint32_t n_chunks,
                                                             int64_t* __restrict__ top, uint32_t* __restrict__ status) {
    __shared__ Stage stg[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t c = blockIdx.x * kWarps + wid;
    if (c >= n_chunks) return;
    const ConcChunk ch = chunks[c];
    const ConcDev dv = devs[ch.dev];
    TopK ta, tk;
    clear_top(ta);
    clear_top(tk);
    uint32_t bad = 0;
    for (uint32_t o = 0; o < ch.n; o += kTile) {
        const int n = static_cast<int>(min(static_cast<uint32_t>(kTile), ch.n - o));
        stage_tile(stg[wid], se, tag, ch.rec0 + o, n, lane);
        for (int i = 0; i < kItems; ++i) {
            const int q = lane * kItems + i;
            if (q < n) {
                const longlong2 r = stg[wid].se[q];
                const uint32_t kind = stg[wid].tag[q] >> 5;
                bad |= (r.y < r.x ? 1u : 0u) | (kind > 4u ? 2u : 0u);
                const int64_t e = min64(r.y, dv.b);
                insert_top(ta, e);
                if (kind == 0u) insert_top(tk, e);
            }
        }
        __syncwarp();
    }
    // reduce the lanes' lists: the last lane of an inclusive scan holds all
    scan_top(ta, lane);
    scan_top(tk, lane);
    bad = __reduce_or_sync(0xFFFFFFFFu, bad);
    if (lane == 31) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            top[static_cast<uint64_t>(c) * 2 * K + i] = ta.v[i];
            top[static_cast<uint64_t>(c) * 2 * K + K + i] = tk.v[i];
        }
        if (bad) atomicOr(status, bad);
    }
}

// --------------------------------------------------- per-device chunk scan
// entering state of each chunk: top-K over all earlier chunks of its device
__global__ void conc_chunk_scan(const ConcDev* __restrict__ devs, uint32_t n_dev, const int64_t* __restrict__ top,
                                int64_t* __restrict__ in) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_dev) return;
    const ConcDev dv = devs[g];
    TopK ra, rk;
    clear_top(ra);
    clear_top(rk);
    for (uint32_t q = 0; q < dv.nchunk; ++q) {
        const uint64_t c = dv.chunk0 + q;
        TopK xa, xk;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            in[c * 2 * K + i] = ra.v[i];
            in[c * 2 * K + K + i] = rk.v[i];
            xa.v[i] = top[c * 2 * K + i];
            xk.v[i] = top[c * 2 * K + K + i];
        }
        merge_top(ra, xa);
        merge_top(rk, xk);
    }
}

// ------------------------------------------------------------- levels
__global__ void __launch_bounds__(kWarps * 32) conc_chunk_levels(const int64_t* __restrict__ se,
                                                                const uint8_t* __restrict__ tag,
                                                                const ConcDev* __restrict__ devs,
                                                                const ConcChunk* __restrict__ chunks,
                                                                uint32_t n_chunks, const int64_t* __restrict__ in,
                                                                int64_t* __restrict__ out,
                                                                uint32_t* __restrict__ status) {
    __shared__ Stage stg[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t c = blockIdx.x * kWarps + wid;
    if (c >= n_chunks) return;
    const ConcChunk ch = chunks[c];
    const ConcDev dv = devs[ch.dev];
    TopK sa, sk;   // state before the current tile
#pragma unroll
    for (int i = 0; i < K; ++i) {
        sa.v[i] = in[static_cast<uint64_t>(c) * 2 * K + i];
        sk.v[i] = in[static_cast<uint64_t>(c) * 2 * K + K + i];
    }
    int64_t acc_a[K], acc_k[K];
#pragma unroll
    for (int i = 0; i < K; ++i) acc_a[i] = acc_k[i] = 0;
    uint32_t bad = 0;
    const uint64_t dev_end = dv.rec0 + dv.n;
    for (uint32_t o = 0; o < ch.n; o += kTile) {
        const int n = static_cast<int>(min(static_cast<uint32_t>(kTile), ch.n - o));
        const uint64_t r0 = ch.rec0 + o;
        stage_tile(stg[wid], se, tag, r0, n, lane);
        if (o > 0 && lane == 0) bad |= se[2 * (r0 - 1)] > se[2 * r0] ? 4u : 0u;
        // start of the record after the tile (clipped), or none
        int64_t after = INT64_MAX;
        if (r0 + n < dev_end) after = max64(se[2 * (r0 + n)], dv.a);
        // lane lists of this tile's ends, scanned across the warp
        TopK la, lk;
        clear_top(la);
        clear_top(lk);
        int64_t s[kItems], e[kItems];
        uint32_t kd[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int q = lane * kItems + i;
            if (q < n) {
                const longlong2 r = stg[wid].se[q];
                s[i] = max64(r.x, dv.a);
                e[i] = max64(min64(r.y, dv.b), s[i]);
                kd[i] = stg[wid].tag[q] >> 5;
                if (q > 0) bad |= stg[wid].se[q - 1].x > r.x ? 4u : 0u;
                insert_top(la, e[i]);
                if (kd[i] == 0u) insert_top(lk, e[i]);
            } else {
                s[i] = e[i] = INT64_MAX;
                kd[i] = 1u;
            }
        }
        scan_top(la, lane);
        scan_top(lk, lane);
        // entering state of this lane = tile state + lanes before it
        TopK xa = shfl_up_top(la, 1), xk = shfl_up_top(lk, 1);
        if (lane == 0) {
            clear_top(xa);
            clear_top(xk);
        }
        merge_top(xa, sa);
        merge_top(xk, sk);
        // next lane's first start (the last lane: the record after the tile)
        int64_t nxt = shfl64(s[0], (lane + 1) & 31);
        if (lane == 31 || (lane + 1) * kItems >= n) nxt = after;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int q = lane * kItems + i;
            if (q < n) {
                insert_top(xa, e[i]);
                if (kd[i] == 0u) insert_top(xk, e[i]);
                const int64_t ns = (i + 1 < kItems && q + 1 < n) ? s[i + 1] : nxt;
                const int64_t hi = min64(ns, dv.b);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    // E_k below s_i (or none: INT64_MIN) contributes nothing;
                    // clamping first keeps the difference from overflowing
                    acc_a[k] += max64(min64(hi, max64(xa.v[k], s[i])) - s[i], 0);
                    acc_k[k] += max64(min64(hi, max64(xk.v[k], s[i])) - s[i], 0);
                }
            }
        }
        // state after the tile: everything up to the last lane
        const TopK ta = shfl_top(la, 31), tk = shfl_top(lk, 31);
        merge_top(sa, ta);
        merge_top(sk, tk);
        __syncwarp();
    }
    if (ch.n > 0 && ch.rec0 > dv.rec0 && lane == 0) bad |= se[2 * (ch.rec0 - 1)] > se[2 * ch.rec0] ? 4u : 0u;
    bad = __reduce_or_sync(0xFFFFFFFFu, bad);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t va = warp_sum64(acc_a[k]);
        const int64_t vk = warp_sum64(acc_k[k]);
        if (lane == 0) {
            if (va) atomic_add64(&out[static_cast<uint64_t>(ch.dev) * 2 * K + k], va);
            if (vk) atomic_add64(&out[static_cast<uint64_t>(ch.dev) * 2 * K + K + k], vk);
        }
    }
    if (lane == 0 && bad) atomicOr(status, bad);
}

}  // namespace

cudaError_t launch_concurrency(const int64_t* se, const uint8_t* tag, const ConcDev* devs, uint32_t n_dev,
                               const ConcChunk* chunks, uint32_t n_chunks, int64_t* top, int64_t* in, int64_t* out,
                               uint32_t* status, cudaStream_t stream) {
    if (n_chunks == 0) return cudaSuccess;
    const uint32_t blocks = (n_chunks + kWarps - 1) / kWarps;
    conc_chunk_top<<<blocks, kWarps * 32, 0, stream>>>(se, tag, devs, chunks, n_chunks, top, status);
    conc_chunk_scan<<<(n_dev + 127) / 128, 128, 0, stream>>>(devs, n_dev, top, in);
    conc_chunk_levels<<<blocks, kWarps * 32, 0, stream>>>(se, tag, devs, chunks, n_chunks, in, out, status);
    return cudaGetLastError();
}

}  // namespace talp
