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
static_assert(K == 8 && kItems == 8, "a lane's list is its 8 records sorted by an 8-input network");

// Sorted-descending list of the K largest ends seen.  Two widths: absolute
// int64 (INT64_MIN: none) for the state carried between tiles and chunks,
// and uint32 offsets from a tile's first clipped start for the tile's own
// work (0: at or before that start, which no later record can use).
template <typename T>
struct TopK {
    T v[K];
};

template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <typename T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }

template <typename T>
__device__ __forceinline__ T none_v();
template <>
__device__ __forceinline__ int64_t none_v<int64_t>() { return INT64_MIN; }
template <>
__device__ __forceinline__ uint32_t none_v<uint32_t>() { return 0u; }

template <typename T>
__device__ __forceinline__ void clear_top(TopK<T>& x) {
#pragma unroll
    for (int i = 0; i < K; ++i) x.v[i] = none_v<T>();
}

// top-K of the union of two sorted-descending lists (result sorted)
template <typename T>
__device__ __forceinline__ void merge_top(TopK<T>& x, const TopK<T>& y) {
#pragma unroll
    for (int i = 0; i < K; ++i) x.v[i] = tmax(x.v[i], y.v[K - 1 - i]);   // bitonic
#pragma unroll
    for (int w = K / 2; w > 0; w >>= 1) {
#pragma unroll
        for (int i = 0; i < K; ++i)
            if ((i & w) == 0) {
                const T hi = tmax(x.v[i], x.v[i + w]), lo = tmin(x.v[i], x.v[i + w]);
                x.v[i] = hi;
                x.v[i + w] = lo;
            }
    }
}

// Sorts 8 values into descending order: the 19-comparator network for 8
// inputs (Knuth, TAOCP vol. 3, 5.3.4), checked on all 2^8 0-1 inputs.
__device__ __forceinline__ void sort8_desc(uint32_t (&v)[8]) {
    constexpr int net[19][2] = {{0, 2}, {1, 3}, {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}, {0, 1}, {2, 3},
                                {4, 5}, {6, 7}, {2, 4}, {3, 5}, {1, 4}, {3, 6}, {1, 2}, {3, 4}, {5, 6}};
#pragma unroll
    for (int c = 0; c < 19; ++c) {
        const uint32_t x = v[net[c][0]], y = v[net[c][1]];
        v[net[c][0]] = x > y ? x : y;
        v[net[c][1]] = x > y ? y : x;
    }
}

template <typename T>
__device__ __forceinline__ void insert_top(TopK<T>& x, T e) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const T hi = tmax(x.v[i], e);
        e = tmin(x.v[i], e);
        x.v[i] = hi;
    }
}

__device__ __forceinline__ uint32_t shfl_up_t(uint32_t v, int d) { return __shfl_up_sync(0xFFFFFFFFu, v, d); }
__device__ __forceinline__ uint32_t shfl_t(uint32_t v, int s) { return __shfl_sync(0xFFFFFFFFu, v, s); }
__device__ __forceinline__ int64_t shfl_t(int64_t v, int s) { return shfl64(v, s); }
__device__ __forceinline__ uint32_t shfl_xor_t(uint32_t v, int m) { return __shfl_xor_sync(0xFFFFFFFFu, v, m); }
__device__ __forceinline__ int64_t shfl_xor_t(int64_t v, int m) { return shfl_xor64(v, m); }

template <typename T>
__device__ __forceinline__ TopK<T> shfl_top(const TopK<T>& x, int src) {
    TopK<T> y;
#pragma unroll
    for (int i = 0; i < K; ++i) y.v[i] = shfl_t(x.v[i], src);
    return y;
}

template <typename T>
__device__ __forceinline__ TopK<T> shfl_up_top(const TopK<T>& x, int d) {
    TopK<T> y;
#pragma unroll
    for (int i = 0; i < K; ++i) y.v[i] = shfl_up_t(x.v[i], d);
    return y;
}

// warp-inclusive scan of top-K lists over lanes
template <typename T>
__device__ __forceinline__ void scan_top(TopK<T>& x, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const TopK<T> y = shfl_up_top(x, d);
        if (lane >= d) merge_top(x, y);
    }
}

// absolute value -> offset from s0 (0 at or before s0), and back
__device__ __forceinline__ uint32_t rel32(int64_t x, int64_t s0) {
    if (x <= s0) return 0u;
    const uint64_t d = static_cast<uint64_t>(x) - static_cast<uint64_t>(s0);   // exact: 0 < d < 2^64
    return d > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(d);
}
// x is at or before s0, or within 2^32 - 1 ns after it
__device__ __forceinline__ bool near32(int64_t x, int64_t s0) {
    return x <= s0 || static_cast<uint64_t>(x) - static_cast<uint64_t>(s0) < 0xFFFFFFFFull;
}
__device__ __forceinline__ void to_abs(TopK<int64_t>& out, const TopK<uint32_t>& x, int64_t s0) {
#pragma unroll
    for (int i = 0; i < K; ++i) out.v[i] = s0 + static_cast<int64_t>(x.v[i]);
}

// One tile of a chunk staged in shared memory: rows of 16 bytes and tags.
// Lane L works on records L * kItems .. L * kItems + kItems - 1, so record q
// sits at (q % kItems) * 33 + q / kItems: the lanes' reads of their i-th
// records are consecutive (no bank conflicts), and so are the staging
// writes of 8 consecutive records.
constexpr int kSlots = kItems * 33;
struct Stage {
    longlong2 se[kSlots];
    uint8_t tag[kSlots];
};

__device__ __forceinline__ int slot(int q) { return (q % kItems) * 33 + q / kItems; }

__device__ __forceinline__ void stage_tile(Stage& st, const int64_t* __restrict__ se, const uint8_t* __restrict__ tag,
                                           uint64_t r0, int n, int lane) {
    for (int q = lane; q < n; q += 32) {
        st.se[slot(q)] = *reinterpret_cast<const longlong2*>(se + 2 * (r0 + q));
        st.tag[slot(q)] = tag[r0 + q];
    }
    __syncwarp();
}

__device__ __forceinline__ longlong2 row_of(const Stage& st, int q) { return st.se[slot(q)]; }
__device__ __forceinline__ uint32_t kind_of(const Stage& st, int q) { return st.tag[slot(q)] >> 5; }

// clipped record q of the stage: start max(s, a), end in [start, b]
__device__ __forceinline__ void clipped(const Stage& st, int q, const ConcDev& dv, int64_t& s, int64_t& e) {
    const longlong2 r = row_of(st, q);
    s = max64(r.x, dv.a);
    e = max64(min64(r.y, dv.b), s);
}

// clipped row
__device__ __forceinline__ void clip_row(const longlong2 r, const ConcDev& dv, int64_t& s, int64_t& e) {
    s = max64(r.x, dv.a);
    e = max64(min64(r.y, dv.b), s);
}

// ------------------------------------------------------------- chunk top-K
// The K largest ends of a chunk do not depend on the order of its records:
// each lane takes every 32nd record straight from memory (coalesced) into
// its own lists, as 32-bit offsets from the chunk's first clipped start
// (every clipped start and end of the chunk is at or after it), and the
// warp merges the 32 lists once.  A chunk whose ends reach 2^32 - 1 ns or
// more past its first start is redone with 64-bit lists.
template <typename T>
__device__ __forceinline__ void warp_merge_top(TopK<T>& x) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        TopK<T> y;
#pragma unroll
        for (int i = 0; i < K; ++i) y.v[i] = shfl_xor_t(x.v[i], m);
        merge_top(x, y);
    }
}

__global__ void __launch_bounds__(kWarps * 32) conc_chunk_top(const int64_t* __restrict__ se,
                                                             const uint8_t* __restrict__ tag,
                                                             const ConcDev* __restrict__ devs,
                                                             const ConcChunk* __restrict__ chunks, uint32_t n_chunks,
                                                             int64_t* __restrict__ top, uint32_t* __restrict__ status) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t c = blockIdx.x * kWarps + wid;
    if (c >= n_chunks) return;
    const ConcChunk ch = chunks[c];
    const ConcDev dv = devs[ch.dev];
    TopK<int64_t> ca, ck;
    clear_top(ca);
    clear_top(ck);
    uint32_t bad = 0;
    if (ch.n > 0) {
        int64_t s0, e0;
        clip_row(*reinterpret_cast<const longlong2*>(se + 2 * ch.rec0), dv, s0, e0);
        TopK<uint32_t> la, lk;
        clear_top(la);
        clear_top(lk);
        bool fits = true;
        for (uint32_t q = lane; q < ch.n; q += 32) {
            const longlong2 r = *reinterpret_cast<const longlong2*>(se + 2 * (ch.rec0 + q));
            const uint32_t kind = tag[ch.rec0 + q] >> 5;
            bad |= (r.y < r.x ? 1u : 0u) | (kind > 4u ? 2u : 0u);
            int64_t s, e;
            clip_row(r, dv, s, e);
            fits &= near32(e, s0);
            const uint32_t re = rel32(e, s0);
            insert_top(la, re);
            if (kind == 0u) insert_top(lk, re);
        }
        if (__all_sync(0xFFFFFFFFu, fits)) {
            warp_merge_top(la);
            warp_merge_top(lk);
            to_abs(ca, la, s0);
            to_abs(ck, lk, s0);
        } else {
            for (uint32_t q = lane; q < ch.n; q += 32) {
                int64_t s, e;
                clip_row(*reinterpret_cast<const longlong2*>(se + 2 * (ch.rec0 + q)), dv, s, e);
                insert_top(ca, e);
                if ((tag[ch.rec0 + q] >> 5) == 0u) insert_top(ck, e);
            }
            warp_merge_top(ca);
            warp_merge_top(ck);
        }
    }
    bad = __reduce_or_sync(0xFFFFFFFFu, bad);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            top[static_cast<uint64_t>(c) * 2 * K + i] = ca.v[i];
            top[static_cast<uint64_t>(c) * 2 * K + K + i] = ck.v[i];
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
    TopK<int64_t> ra, rk;
    clear_top(ra);
    clear_top(rk);
    for (uint32_t q = 0; q < dv.nchunk; ++q) {
        const uint64_t c = dv.chunk0 + q;
        TopK<int64_t> xa, xk;
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
__global__ void __launch_bounds__(kWarps * 32, 2) conc_chunk_levels(const int64_t* __restrict__ se,
                                                                const uint8_t* __restrict__ tag,
                                                                const ConcDev* __restrict__ devs,
                                                                const ConcChunk* __restrict__ chunks,
                                                                uint32_t n_chunks, const int64_t* __restrict__ in,
                                                                int64_t* __restrict__ out,
                                                                uint32_t* __restrict__ status) {
    __shared__ Stage stg[kWarps];
    __shared__ unsigned long long s_acc[kWarps][2 * K];   // the warp's level sums of its chunk
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t c = blockIdx.x * kWarps + wid;
    if (c >= n_chunks) return;
    const ConcChunk ch = chunks[c];
    const ConcDev dv = devs[ch.dev];
    if (lane < 2 * K) s_acc[wid][lane] = 0;
    __syncwarp();
    TopK<int64_t> sa, sk;   // state before the current tile (warp-uniform)
#pragma unroll
    for (int i = 0; i < K; ++i) {
        sa.v[i] = in[static_cast<uint64_t>(c) * 2 * K + i];
        sk.v[i] = in[static_cast<uint64_t>(c) * 2 * K + K + i];
    }
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
        int64_t s0, e0;
        clipped(stg[wid], 0, dv, s0, e0);
        // offsets from s0: the tile's records, the entering state, the bounds
        uint32_t s[kItems], e[kItems];
        uint32_t kmask = 0;
        bool fits = true;
        // the lane's own top-K lists: its kItems == K ends sorted (0 = none)
        TopK<uint32_t> la, lk;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int q = lane * kItems + i;
            s[i] = e[i] = 0xFFFFFFFFu;
            la.v[i] = lk.v[i] = 0u;
            if (q < n) {
                int64_t sa64, ea64;
                clipped(stg[wid], q, dv, sa64, ea64);
                if (q > 0) bad |= row_of(stg[wid], q - 1).x > row_of(stg[wid], q).x ? 4u : 0u;
                fits &= near32(ea64, s0);
                s[i] = rel32(sa64, s0);
                e[i] = rel32(ea64, s0);
                const bool isK = kind_of(stg[wid], q) == 0u;
                kmask |= isK ? 1u << i : 0u;
                la.v[i] = e[i];
                lk.v[i] = isK ? e[i] : 0u;
            }
        }
        sort8_desc(la.v);
        sort8_desc(lk.v);
#pragma unroll
        for (int i = 0; i < K; ++i) fits &= near32(sa.v[i], s0) && near32(sk.v[i], s0);
        if (__all_sync(0xFFFFFFFFu, fits)) {
            TopK<uint32_t> ta, tk;   // entering state as offsets
#pragma unroll
            for (int i = 0; i < K; ++i) {
                ta.v[i] = rel32(sa.v[i], s0);
                tk.v[i] = rel32(sk.v[i], s0);
            }
            scan_top(la, lane);
            scan_top(lk, lane);
            TopK<uint32_t> xa = shfl_up_top(la, 1), xk = shfl_up_top(lk, 1);
            if (lane == 0) {
                clear_top(xa);
                clear_top(xk);
            }
            merge_top(xa, ta);
            merge_top(xk, tk);
            // a lane's gaps in the tile are disjoint and lie within 2^32 - 1 ns
            // of s0, so its level sums of the tile fit 32 bits.  The level-k
            // time of a gap [s, hi) is min(max(E_k, s), max(hi, s)) - s; the
            // s terms are summed once (S) and taken off at the end, which is
            // exact in wrapping 32-bit arithmetic because the results fit.
            uint32_t acc_a[K], acc_k[K], S = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) acc_a[k] = acc_k[k] = 0;
            const uint32_t bnd = rel32(dv.b, s0);
            uint32_t nxt = shfl_t(s[0], (lane + 1) & 31);
            if (lane == 31 || (lane + 1) * kItems >= n) nxt = rel32(after, s0);
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                const int q = lane * kItems + i;
                if (q < n) {
                    insert_top(xa, e[i]);
                    if (kmask & (1u << i)) insert_top(xk, e[i]);
                    const uint32_t ns = (i + 1 < kItems && q + 1 < n) ? s[i + 1] : nxt;
                    // the gap [s_i, min(next start, window end)) at level k
                    // lasts until E_k
                    const uint32_t hc = tmax(tmin(ns, bnd), s[i]);
                    S += s[i];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        acc_a[k] += tmin(tmax(xa.v[k], s[i]), hc);
                        acc_k[k] += tmin(tmax(xk.v[k], s[i]), hc);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                acc_a[k] -= S;
                acc_k[k] -= S;
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {   // warp sums in 16-bit halves (no overflow)
                const uint32_t al = __reduce_add_sync(0xFFFFFFFFu, acc_a[k] & 0xFFFFu);
                const uint32_t ah = __reduce_add_sync(0xFFFFFFFFu, acc_a[k] >> 16);
                const uint32_t kl = __reduce_add_sync(0xFFFFFFFFu, acc_k[k] & 0xFFFFu);
                const uint32_t kh = __reduce_add_sync(0xFFFFFFFFu, acc_k[k] >> 16);
                if (lane == 0) {
                    s_acc[wid][k] += (static_cast<unsigned long long>(ah) << 16) + al;
                    s_acc[wid][K + k] += (static_cast<unsigned long long>(kh) << 16) + kl;
                }
            }
            // state after the tile: the entering state and every record of it
            merge_top(la, ta);
            merge_top(lk, tk);
            to_abs(sa, shfl_top(la, 31), s0);
            to_abs(sk, shfl_top(lk, 31), s0);
        } else {
            // a tile spanning 2^32 ns or more: lane 0 walks it in 64 bits
            if (lane == 0) {
                for (int q = 0; q < n; ++q) {
                    int64_t sq, eq;
                    clipped(stg[wid], q, dv, sq, eq);
                    insert_top(sa, eq);
                    const bool isK = kind_of(stg[wid], q) == 0u;
                    if (isK) insert_top(sk, eq);
                    int64_t ns = after;
                    if (q + 1 < n) {
                        int64_t s1, e1;
                        clipped(stg[wid], q + 1, dv, s1, e1);
                        ns = s1;
                    }
                    const int64_t hi = min64(ns, dv.b);
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        s_acc[wid][k] += static_cast<unsigned long long>(max64(min64(hi, max64(sa.v[k], sq)) - sq, 0));
                        s_acc[wid][K + k] +=
                            static_cast<unsigned long long>(max64(min64(hi, max64(sk.v[k], sq)) - sq, 0));
                    }
                }
            }
            sa = shfl_top(sa, 0);
            sk = shfl_top(sk, 0);
        }
        __syncwarp();
    }
    if (ch.n > 0 && ch.rec0 > dv.rec0 && lane == 0) bad |= se[2 * (ch.rec0 - 1)] > se[2 * ch.rec0] ? 4u : 0u;
    bad = __reduce_or_sync(0xFFFFFFFFu, bad);
    __syncwarp();
    if (lane < 2 * K) {
        const int64_t v = static_cast<int64_t>(s_acc[wid][lane]);
        if (v) atomic_add64(&out[static_cast<uint64_t>(ch.dev) * 2 * K + lane], v);
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
