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
// A device's record list is cut into chunks, each walked tile by tile by one
// warp.  A main pass walks every chunk as if nothing ran into it and leaves
// the chunk's exit state (its largest ends still running after its last
// start); a per-device scan of those gives each chunk its true entering
// state; a fix-up pass walks again, with both entering states, the leading
// tiles of the chunks into which earlier ends still run, and adds the
// difference.  Top-K merges are bitonic (elementwise max against the
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
__device__ __forceinline__ int64_t shfl_up_t(int64_t v, int d) { return shfl_up64(v, d); }
__device__ __forceinline__ uint32_t shfl_t(uint32_t v, int s) { return __shfl_sync(0xFFFFFFFFu, v, s); }
__device__ __forceinline__ int64_t shfl_t(int64_t v, int s) { return shfl64(v, s); }

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

// absolute value -> offset from s0 (0 at or before s0)
__device__ __forceinline__ uint32_t rel32(int64_t x, int64_t s0) {
    if (x <= s0) return 0u;
    const uint64_t d = static_cast<uint64_t>(x) - static_cast<uint64_t>(s0);   // exact: 0 < d < 2^64
    return d > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(d);
}
// x is at or before s0, or within 2^32 - 1 ns after it
__device__ __forceinline__ bool near32(int64_t x, int64_t s0) {
    return x <= s0 || static_cast<uint64_t>(x) - static_cast<uint64_t>(s0) < 0xFFFFFFFFull;
}

// One tile of a chunk staged in shared memory: rows of 16 bytes and tags.
// Lane L works on records L * kItems .. L * kItems + kItems - 1, so record q
// sits at (q % kItems) * 33 + q / kItems: the lanes' reads of their i-th
// records are consecutive (no bank conflicts), and so are the staging
// writes of 8 consecutive records.  The tags arrive as the aligned 4-byte
// words that hold the tile's tag bytes (each word holds at least one of
// them, so it lies in mapped memory); byte q is at toff + q.
constexpr int kSlots = kItems * 33;
constexpr int kTagWords = kTile / 4 + 2;
struct Stage {
    longlong2 se[kSlots];
    uint32_t tagw[kTagWords];
};

__device__ __forceinline__ int slot(int q) { return (q % kItems) * 33 + q / kItems; }

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copies of one tile (records r0 .. r0 + n - 1) into a stage, issued by
// every lane as one commit group; they land while the warp works on the
// tile before.
__device__ __forceinline__ void issue_tile(Stage& st, const int64_t* __restrict__ se, const uint8_t* __restrict__ tag,
                                           uint64_t r0, int n, int lane) {
    // record lane + 32 j sits at slot (lane % 8) * 33 + lane / 8 + 4 j
    longlong2* dst = &st.se[slot(lane)];
    const int64_t* src = se + 2 * (r0 + lane);
#pragma unroll
    for (int j = 0; j < kItems; ++j)
        if (lane + 32 * j < n) cp_async16(dst + 4 * j, src + 64 * j);
    const uintptr_t A = reinterpret_cast<uintptr_t>(tag + r0);
    const uintptr_t w0 = A & ~static_cast<uintptr_t>(3);
    const int nw = static_cast<int>((A + static_cast<uintptr_t>(n) + 3 - w0) >> 2);
    for (int w = lane; w < nw; w += 32) cp_async4(&st.tagw[w], reinterpret_cast<const void*>(w0 + 4u * w));
    cp_async_commit();
}

__device__ __forceinline__ longlong2 row_of(const Stage& st, int q) { return st.se[slot(q)]; }
__device__ __forceinline__ uint32_t kind_of(const Stage& st, int toff, int q) {
    return reinterpret_cast<const uint8_t*>(st.tagw)[toff + q] >> 5;
}

// clipped record q of the stage: start max(s, a), end in [start, b]
__device__ __forceinline__ void clipped(const Stage& st, int q, const ConcDev& dv, int64_t& s, int64_t& e) {
    const longlong2 r = row_of(st, q);
    s = max64(r.x, dv.a);
    e = max64(min64(r.y, dv.b), s);
}


// --------------------------------------------------- per-device chunk scan
// Entering state of each chunk: the top-K over all earlier chunks of its
// device.  One warp per device, 32 chunks at a time: a warp scan of the
// chunks' lists, merged with the carry of the chunks before.
constexpr int kScanWarps = 4;

__global__ void __launch_bounds__(kScanWarps * 32) conc_chunk_scan(const ConcDev* __restrict__ devs, uint32_t n_dev,
                                                                  const int64_t* __restrict__ top,
                                                                  int64_t* __restrict__ in) {
    const int lane = threadIdx.x & 31;
    const uint32_t g = blockIdx.x * kScanWarps + (threadIdx.x >> 5);
    if (g >= n_dev) return;
    const ConcDev dv = devs[g];
    TopK<int64_t> ca, ck;   // carry: every chunk before the current group
    clear_top(ca);
    clear_top(ck);
    for (uint32_t q0 = 0; q0 < dv.nchunk; q0 += 32) {
        const uint32_t q = q0 + lane;
        const uint64_t c = static_cast<uint64_t>(dv.chunk0) + q;
        TopK<int64_t> xa, xk;
        clear_top(xa);
        clear_top(xk);
        if (q < dv.nchunk) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                xa.v[i] = top[c * 2 * K + i];
                xk.v[i] = top[c * 2 * K + K + i];
            }
        }
        scan_top(xa, lane);
        scan_top(xk, lane);
        TopK<int64_t> ea = shfl_up_top(xa, 1), ek = shfl_up_top(xk, 1);
        if (lane == 0) {
            clear_top(ea);
            clear_top(ek);
        }
        merge_top(ea, ca);
        merge_top(ek, ck);
        if (q < dv.nchunk) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                in[c * 2 * K + i] = ea.v[i];
                in[c * 2 * K + K + i] = ek.v[i];
            }
        }
        merge_top(ca, shfl_top(xa, 31));
        merge_top(ck, shfl_top(xk, 31));
    }
}

// ------------------------------------------------------------- levels
// The state carried from tile to tile (the K largest ends before the tile
// that may still be running at its start; ends known to have finished may
// be missing, as they add nothing) is kept as 32-bit offsets from the
// previous tile's first start
// and rebased on the next tile's with one max and one subtraction per entry
// (an entry at or before the new base becomes 0: no later start can use
// it).  Only when a tile had to take the int64 path does the state live as
// int64 in shared memory until a tile converts it back.
//
// In a lane's walk the K = 8 list is split in two: the 4 largest ends (every
// record updates them) and the next 4, which an end joins only when the top
// 4 push it out while it is still running at the record's start (a
// concurrency of 5 or more, rare); levels 5-8 are added only for records at
// which some lane of the warp has such an end.
// Top 4 of two sorted-descending lists of 4, into the first 4 entries of x:
// elementwise max against the reversed list, then a bitonic half-cleaner
// cascade.
__device__ __forceinline__ void merge4(uint32_t* x, const uint32_t (&y)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = tmax(x[i], y[3 - i]);
#pragma unroll
    for (int w = 2; w > 0; w >>= 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if ((i & w) == 0) {
                const uint32_t hi = tmax(x[i], x[i + w]), lo = tmin(x[i], x[i + w]);
                x[i] = hi;
                x[i + w] = lo;
            }
    }
}

// Insertion of e into a sorted-descending list of 4, e left as the value
// pushed out.  Entry k of the result is max(x[k], min(x[k-1], e)) -- x[k]
// above e's place, e at it, x[k-1] below it -- so all four come out in two
// dependent steps instead of a chain through the list.
__device__ __forceinline__ void ins4(uint32_t (&x)[4], uint32_t& e) {
    const uint32_t out = tmin(x[3], e);
    x[3] = tmax(x[3], tmin(x[2], e));
    x[2] = tmax(x[2], tmin(x[1], e));
    x[1] = tmax(x[1], tmin(x[0], e));
    x[0] = tmax(x[0], e);
    e = out;
}

template <bool FIX>
__global__ void __launch_bounds__(kWarps * 32, 2) conc_chunk_levels(const int64_t* __restrict__ se,
                                                                const uint8_t* __restrict__ tag,
                                                                const ConcDev* __restrict__ devs,
                                                                const ConcChunk* __restrict__ chunks,
                                                                uint32_t n_chunks, const int64_t* __restrict__ in,
                                                                int64_t* __restrict__ top, int64_t* __restrict__ snap,
                                                                int64_t* __restrict__ out,
                                                                uint32_t* __restrict__ status) {
    // per warp: two stages (the tile being worked on and the next one in
    // flight), then the level sums and the int64 state of every warp
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    Stage* stg = reinterpret_cast<Stage*>(smem) + 2 * wid;
    unsigned long long* s_acc =
        reinterpret_cast<unsigned long long*>(smem + sizeof(Stage) * 2 * kWarps) + wid * 2 * K;   // level sums
    int64_t* s_st = reinterpret_cast<int64_t*>(smem + sizeof(Stage) * 2 * kWarps) + (kWarps + wid) * 2 * K;
    unsigned long long* s_acc2 =
        reinterpret_cast<unsigned long long*>(smem + sizeof(Stage) * 2 * kWarps) + (2 * kWarps + wid) * 2 * K;
    const uint32_t c = blockIdx.x * kWarps + wid;
    if (c >= n_chunks) return;
    const ConcChunk ch = chunks[c];
    const ConcDev dv = devs[ch.dev];
    // FIX: the largest end running into the chunk (its true entering state is
    // sorted); a chunk it does not reach past its first start needs nothing
    const int64_t E1 = FIX ? in[static_cast<uint64_t>(c) * 2 * K] : INT64_MIN;
    if (FIX && (ch.n == 0 || E1 <= max64(se[2 * ch.rec0], dv.a))) return;
    uint32_t bad = 0;
    // state before the current tile (warp-uniform): offsets from sbase when
    // rel, else s_st
    bool rel = false;
    int64_t sbase = 0;
    uint32_t ra[K], rk[K];
    const uint64_t dev_end = dv.rec0 + dv.n;
    // The main pass keeps its level sums after a chunk's first and second
    // tiles (snap[c][0..1]).  When the fix-up's walk with the true state ends
    // within those tiles, the same walk with no entering state is the main
    // pass's and its sums are taken from snap instead of a second walk.
    uint32_t walked = 0;   // tiles the current pass has walked
    bool use_snap = false;
    for (int pass = 0; pass < (FIX ? 2 : 1); ++pass) {
        walked = 0;
        unsigned long long* acc = pass ? s_acc2 : s_acc;
        if (ch.n > 0)
            issue_tile(stg[0], se, tag, ch.rec0, static_cast<int>(min(static_cast<uint32_t>(kTile), ch.n)), lane);
        if (lane < 2 * K) {
            acc[lane] = 0;
            // entering state: none (main pass), the true one (fix-up, pass 0)
            s_st[lane] = FIX && pass == 0 ? in[static_cast<uint64_t>(c) * 2 * K + lane] : INT64_MIN;
        }
        __syncwarp();
        rel = false;
        sbase = 0;
#pragma unroll
        for (int i = 0; i < K; ++i) ra[i] = rk[i] = 0u;
        int64_t last_x = INT64_MIN;   // the previous tile's last start (order check)
        // start of the record after a tile (clipped), or none: loaded one tile
        // ahead, so that its latency hides behind a tile's work
        int64_t after_nx = INT64_MAX;
        {
            const uint64_t p = ch.rec0 + min(static_cast<uint32_t>(kTile), ch.n);
            if (p < dev_end) after_nx = max64(se[2 * p], dv.a);
        }
        for (uint32_t o = 0, t = 0; o < ch.n; o += kTile, ++t) {
            const int n = static_cast<int>(min(static_cast<uint32_t>(kTile), ch.n - o));
            const uint64_t r0 = ch.rec0 + o;
            const int64_t after = after_nx;
            if (o + kTile < ch.n) {
                const uint64_t p = r0 + kTile + min(static_cast<uint32_t>(kTile), ch.n - o - kTile);
                after_nx = p < dev_end ? max64(se[2 * p], dv.a) : INT64_MAX;
            }
            if (o + kTile < ch.n) {
                issue_tile(stg[(t + 1) & 1], se, tag, r0 + kTile,
                           static_cast<int>(min(static_cast<uint32_t>(kTile), ch.n - o - kTile)), lane);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();
            const Stage& S = stg[t & 1];
            const int toff = static_cast<int>(reinterpret_cast<uintptr_t>(tag + r0) & 3u);
            const int64_t x0 = row_of(S, 0).x, xl = row_of(S, n - 1).x;
            if (lane == 0) bad |= last_x > x0 ? 4u : 0u;
            last_x = xl;
            const int64_t s0 = max64(x0, dv.a);
            if (FIX && s0 >= E1) {   // both entering states agree on every end running from here on
                cp_async_wait<0>();
                __syncwarp();
                break;
            }
            // the entering state as offsets from s0
            TopK<uint32_t> ta, tk;
            bool fits = true;
            if (rel) {
                const int64_t d = s0 - sbase;
                if (d >= 0 && d <= 0xFFFFFFFFll) {
                    const uint32_t d32 = static_cast<uint32_t>(d);
#pragma unroll
                    for (int i = 0; i < K; ++i) {
                        ta.v[i] = tmax(ra[i], d32) - d32;
                        tk.v[i] = tmax(rk[i], d32) - d32;
                    }
                } else {   // every entry at or before s0 (or records out of order, reported)
                    clear_top(ta);
                    clear_top(tk);
                }
            } else {
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    const int64_t xa = s_st[i], xk = s_st[K + i];
                    fits &= near32(xa, s0) && near32(xk, s0);
                    ta.v[i] = rel32(xa, s0);
                    tk.v[i] = rel32(xk, s0);
                }
            }
            // the tile's records as offsets from s0.  A tile that starts inside
            // the window needs no start clip, and ends are clipped to b only:
            // an end below its start (a record after b) is at or before every
            // later start, so it only ever contributes 0 -- as the gap bound
            // min(next start, b) already makes the gaps after b empty.
            uint32_t s[kItems], e[kItems];
            uint32_t kmask = 0;
            TopK<uint32_t> la, lk;   // the lane's own K ends, sorted (0 = none)
            const bool plain = x0 >= dv.a && x0 < dv.b && static_cast<uint64_t>(xl - x0) < 0xFFFFFFFFull;
            if (plain) {
                uint32_t hib = 0;
                int64_t prev = lane > 0 ? row_of(S, lane * kItems - 1).x : x0;
                // record i of the lane (q = its tile index)
                auto item = [&](int i, int q) {
                    const longlong2 r = row_of(S, q);
                    bad |= (prev > r.x ? 4u : 0u) | (r.y < r.x ? 1u : 0u);
                    prev = r.x;
                    const int64_t de = min64(r.y, dv.b) - s0;
                    hib |= static_cast<uint32_t>(static_cast<uint64_t>(de) >> 32);
                    s[i] = static_cast<uint32_t>(r.x) - static_cast<uint32_t>(s0);
                    e[i] = static_cast<uint32_t>(de);
                    const uint32_t kd = kind_of(S, toff, q);
                    bad |= kd > 4u ? 2u : 0u;
                    const bool isK = kd == 0u;
                    kmask |= isK ? 1u << i : 0u;
                    la.v[i] = e[i];
                    lk.v[i] = isK ? e[i] : 0u;
                };
#pragma unroll
                for (int i = 0; i < kItems; ++i) {
                    const int q = lane * kItems + i;
                    s[i] = e[i] = 0xFFFFFFFFu;
                    la.v[i] = lk.v[i] = 0u;
                    if (q < n) item(i, q);
                }
                fits &= hib == 0;
            } else {
#pragma unroll
                for (int i = 0; i < kItems; ++i) {
                    const int q = lane * kItems + i;
                    s[i] = e[i] = 0xFFFFFFFFu;
                    la.v[i] = lk.v[i] = 0u;
                    if (q < n) {
                        int64_t sa64, ea64;
                        clipped(S, q, dv, sa64, ea64);
                        const longlong2 r = row_of(S, q);
                        if (q > 0) bad |= row_of(S, q - 1).x > r.x ? 4u : 0u;
                        bad |= r.y < r.x ? 1u : 0u;
                        fits &= near32(ea64, s0);
                        s[i] = rel32(sa64, s0);
                        e[i] = rel32(ea64, s0);
                        const uint32_t kd = kind_of(S, toff, q);
                        bad |= kd > 4u ? 2u : 0u;
                        const bool isK = kd == 0u;
                        kmask |= isK ? 1u << i : 0u;
                        la.v[i] = e[i];
                        lk.v[i] = isK ? e[i] : 0u;
                    }
                }
            }
            sort8_desc(la.v);
            sort8_desc(lk.v);
            if (__all_sync(0xFFFFFFFFu, fits)) {
                // A lane needs from the lanes before it only the ends still
                // running at its first start th (a lane without records: at the
                // next tile's first start).  With pm the largest end of lanes
                // 0 .. L (kernel ends are among them), lane L looks back at lane
                // L - d only while pm(L - d) > th: usually the previous lane or
                // two.  The ends at or before th it skips contribute nothing to
                // its records, nor to any later lane.
                const uint32_t aft = rel32(after, s0);
                const uint32_t th = lane * kItems < n ? s[0] : aft;
                uint32_t pm = la.v[0];
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, pm, d);
                    if (lane >= d) pm = tmax(pm, y);
                }
                // The lanes looked back at and the entering state usually hold
                // at most 4 ends still running at th between them; then their
                // top 4 lists carry all of those (a kernel end running at th is
                // one of them), and ends at or before th add nothing to this
                // lane's gaps nor to the exit state.  Only when 5 or more run
                // does the warp merge the full lists.
                TopK<uint32_t> xa, xk;
                clear_top(xa);
                clear_top(xk);
                // ends of the entering state and of the looked-back lanes
                // running at th (the first 5 of each list counted)
                uint32_t run = 0;
#pragma unroll
                for (int i = 0; i < 5; ++i) run += ta.v[i] > th ? 1u : 0u;
                for (int d = 1; d < 32; ++d) {
                    const uint32_t pd = __shfl_up_sync(0xFFFFFFFFu, pm, d);
                    const bool need = lane >= d && pd > th;
                    if (!__any_sync(0xFFFFFFFFu, need)) break;
                    uint32_t ya[4], yk[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        ya[i] = __shfl_up_sync(0xFFFFFFFFu, la.v[i], d);
                        yk[i] = __shfl_up_sync(0xFFFFFFFFu, lk.v[i], d);
                    }
                    const uint32_t y4 = __shfl_up_sync(0xFFFFFFFFu, la.v[4], d);
                    if (need) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) run += ya[i] > th ? 1u : 0u;
                        run += y4 > th ? 1u : 0u;
                        merge4(xa.v, ya);
                        merge4(xk.v, yk);
                    }
                }
                if (__any_sync(0xFFFFFFFFu, run > 4)) {
                    clear_top(xa);
                    clear_top(xk);
                    for (int d = 1; d < 32; ++d) {
                        const uint32_t pd = __shfl_up_sync(0xFFFFFFFFu, pm, d);
                        const bool need = lane >= d && pd > th;
                        if (!__any_sync(0xFFFFFFFFu, need)) break;
                        const TopK<uint32_t> ya = shfl_up_top(la, d), yk = shfl_up_top(lk, d);
                        if (need) {
                            merge_top(xa, ya);
                            merge_top(xk, yk);
                        }
                    }
                    merge_top(xa, ta);
                    merge_top(xk, tk);
                } else {
                    uint32_t t4a[4], t4k[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        t4a[i] = ta.v[i];
                        t4k[i] = tk.v[i];
                    }
                    merge4(xa.v, t4a);
                    merge4(xk.v, t4k);
                }
                // a lane's gaps in the tile are disjoint and lie within 2^32 - 1 ns
                // of s0, so its level sums of the tile -- and the warp's, whose
                // gaps are disjoint too -- fit 32 bits.  The level-k time of a gap
                // [s, hi) is min(max(E_k, s), max(hi, s)) - s; the s terms are
                // summed once (S, and SH for the gaps where levels 5-8 are added)
                // and taken off at the end, exact in wrapping 32-bit arithmetic
                // because the results fit.
                uint32_t ma[4], oa[4], mk[4], ok[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    ma[i] = xa.v[i];
                    oa[i] = xa.v[4 + i];
                    mk[i] = xk.v[i];
                    ok[i] = xk.v[4 + i];
                }
                uint32_t acc_a[K], acc_k[K], S = 0, SH = 0;
#pragma unroll
                for (int k = 0; k < K; ++k) acc_a[k] = acc_k[k] = 0;
                const uint32_t bnd = rel32(dv.b, s0);
                uint32_t nxt = shfl_t(s[0], (lane + 1) & 31);
                if (lane == 31 || (lane + 1) * kItems >= n) nxt = aft;
#pragma unroll
                for (int i = 0; i < kItems; ++i) {
                    const int q = lane * kItems + i;
                    const bool v = q < n;
                    const uint32_t ns = (i + 1 < kItems && q + 1 < n) ? s[i + 1] : nxt;
                    // the gap [s_i, min(next start, window end)) at level k
                    // lasts until E_k
                    const uint32_t hc = tmax(tmin(ns, bnd), s[i]);
                    if (v) {
                        uint32_t ev = e[i];
                        ins4(ma, ev);
                        if (ev > s[i]) ins4(oa, ev);   // a 5th end still running
                        if (kmask & (1u << i)) {
                            uint32_t ek = e[i];
                            ins4(mk, ek);
                            if (ek > s[i]) ins4(ok, ek);
                        }
                        S += s[i];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            acc_a[k] += tmin(tmax(ma[k], s[i]), hc);
                            acc_k[k] += tmin(tmax(mk[k], s[i]), hc);
                        }
                    }
                    if (__any_sync(0xFFFFFFFFu, v && tmax(oa[0], ok[0]) > s[i])) {
                        if (v) {
                            SH += s[i];
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                acc_a[4 + k] += tmin(tmax(oa[k], s[i]), hc);
                                acc_k[4 + k] += tmin(tmax(ok[k], s[i]), hc);
                            }
                        }
                    }
                }
                // lane k < 2K adds level sum k (one shared-memory update per lane,
                // side by side)
                uint32_t mine = 0;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const uint32_t sub = k < 4 ? S : SH;
                    const uint32_t wa = __reduce_add_sync(0xFFFFFFFFu, acc_a[k] - sub);
                    const uint32_t wk = __reduce_add_sync(0xFFFFFFFFu, acc_k[k] - sub);
                    mine = lane == k ? wa : mine;
                    mine = lane == K + k ? wk : mine;
                }
                if (lane < 2 * K) acc[lane] += mine;
                // state after the tile: lane 31's lists after its walk hold every
                // end still running at its last start (or, without records, at
                // the next tile's first start), which covers every end running at
                // the next tile's first start
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    ra[i] = shfl_t(ma[i], 31);
                    ra[4 + i] = shfl_t(oa[i], 31);
                    rk[i] = shfl_t(mk[i], 31);
                    rk[4 + i] = shfl_t(ok[i], 31);
                }
                sbase = s0;
                rel = true;
            } else {
                // a tile spanning 2^32 ns or more: lane 0 walks it in 64 bits
                if (lane == 0) {
                    TopK<int64_t> sa, sk;
#pragma unroll
                    for (int i = 0; i < K; ++i) {
                        if (rel) {
                            sa.v[i] = ra[i] ? sbase + static_cast<int64_t>(ra[i]) : INT64_MIN;
                            sk.v[i] = rk[i] ? sbase + static_cast<int64_t>(rk[i]) : INT64_MIN;
                        } else {
                            sa.v[i] = s_st[i];
                            sk.v[i] = s_st[K + i];
                        }
                    }
                    for (int q = 0; q < n; ++q) {
                        int64_t sq, eq;
                        clipped(S, q, dv, sq, eq);
                        insert_top(sa, eq);
                        const bool isK = kind_of(S, toff, q) == 0u;
                        if (isK) insert_top(sk, eq);
                        int64_t ns = after;
                        if (q + 1 < n) {
                            int64_t s1, e1;
                            clipped(S, q + 1, dv, s1, e1);
                            ns = s1;
                        }
                        const int64_t hi = min64(ns, dv.b);
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            acc[k] += static_cast<unsigned long long>(max64(min64(hi, max64(sa.v[k], sq)) - sq, 0));
                            acc[K + k] +=
                                static_cast<unsigned long long>(max64(min64(hi, max64(sk.v[k], sq)) - sq, 0));
                        }
                    }
#pragma unroll
                    for (int i = 0; i < K; ++i) {
                        s_st[i] = sa.v[i];
                        s_st[K + i] = sk.v[i];
                    }
                }
                rel = false;
            }
            __syncwarp();
            if (!FIX && t < 2 && lane < 2 * K)
                snap[(static_cast<uint64_t>(c) * 2 + t) * 2 * K + lane] = static_cast<int64_t>(acc[lane]);
            ++walked;
        }
        if (FIX && pass == 0 && walked >= 1 && walked <= 2) {
            use_snap = true;
            break;
        }
    }   // passes
    if (!FIX && ch.n > 0 && ch.rec0 > dv.rec0 && lane == 0) bad |= se[2 * (ch.rec0 - 1)] > se[2 * ch.rec0] ? 4u : 0u;
    bad = __reduce_or_sync(0xFFFFFFFFu, bad);
    __syncwarp();
    if (lane < 2 * K) {
        // main pass: the level sums with no entering state, and the state
        // after the chunk for the per-device scan; fix-up: the difference the
        // true entering state makes
        int64_t v = static_cast<int64_t>(s_acc[lane]);
        if (FIX)
            v -= use_snap ? snap[(static_cast<uint64_t>(c) * 2 + walked - 1) * 2 * K + lane]
                          : static_cast<int64_t>(s_acc2[lane]);
        if (v) atomic_add64(&out[static_cast<uint64_t>(ch.dev) * 2 * K + lane], v);
        if (!FIX) {
            int64_t x = s_st[lane];
            if (rel) {
                uint32_t r = 0;
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    r = lane == i ? ra[i] : r;
                    r = lane == K + i ? rk[i] : r;
                }
                x = r ? sbase + static_cast<int64_t>(r) : INT64_MIN;
            }
            top[static_cast<uint64_t>(c) * 2 * K + lane] = x;
        }
    }
    if (lane == 0 && bad) atomicOr(status, bad);
}

}  // namespace

cudaError_t launch_concurrency(const int64_t* se, const uint8_t* tag, const ConcDev* devs, uint32_t n_dev,
                               const ConcChunk* chunks, uint32_t n_chunks, int64_t* top, int64_t* in, int64_t* snap,
                               int64_t* out, uint32_t* status, cudaStream_t stream) {
    if (n_chunks == 0) return cudaSuccess;
    const uint32_t blocks = (n_chunks + kWarps - 1) / kWarps;
    constexpr int kSmem = static_cast<int>(sizeof(Stage)) * 2 * kWarps + 3 * kWarps * 2 * K * 8;
    static bool attr_set = false;   // set once per process, before the first launch
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(conc_chunk_levels<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conc_chunk_levels<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    // main pass (no entering state; each chunk's state after it into top),
    // per-device scan (top -> in), fix-up of the chunks' leading tiles
    conc_chunk_levels<false><<<blocks, kWarps * 32, kSmem, stream>>>(se, tag, devs, chunks, n_chunks, nullptr, top,
                                                                     snap, out, status);
    conc_chunk_scan<<<(n_dev + kScanWarps - 1) / kScanWarps, kScanWarps * 32, 0, stream>>>(devs, n_dev, top, in);
    conc_chunk_levels<true><<<blocks, kWarps * 32, kSmem, stream>>>(se, tag, devs, chunks, n_chunks, in, nullptr,
                                                                    snap, out, status);
    return cudaGetLastError();
}

}  // namespace talp
