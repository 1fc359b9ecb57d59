// Device twin of tracegen/igen.py: a counter-based synthetic trace generator.
//
// Test and benchmark infrastructure only (it makes inputs; it computes
// nothing of the reduction).  Every value is a pure function of (lane key,
// slot index, draw number) through the SplitMix64 output function (Steele,
// Lea and Flood, "Fast splittable pseudorandom number generators", 2014),
// and durations come from integer inverse-CDF tables built on the host, so
// the numpy twin reproduces any lane bit for bit.
//
// Lane layouts (all int64 ns, 16-byte {start, end} rows):
//   device lane, E events: S = (7E + 5) / 10 kernel slots back to back,
//     slot j = kernel [ks_j, ks_j + kd_j) then a gap; ks_0 = t0.  Slot j
//     carries one copy iff ((j+1) C) / S - (j C) / S == 1 (C = E - S); the
//     copy starts inside the kernel (30%) or inside the gap after it, so a
//     lane comes out in start order.  Event index of slot j's kernel:
//     j + (j C) / S, its copy right after.
//   host lane, H intervals + 1: back-to-back intervals from t0 with
//     exponential durations by state, then one offload interval up to the
//     rank's end T (written by igen_pad once every lane's end is known).
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 8;
constexpr int kChunk = kThreads * kPer;   // slots per chunk

struct Lane {                 // 64 bytes, mirrored by igen.py
    uint64_t key;
    uint64_t out;             // first output row (device rows or host rows)
    uint64_t n;               // device: events E; host: intervals H
    int64_t t0;
    int64_t mean_gap;         // device: mean kernel gap (ns)
    uint32_t chunk0;          // first chunk of the lane
    uint32_t work_milli;      // device: kernel duration factor x 1000
    uint8_t is_host, law, n_kstreams, copy_stream0, n_cstreams, pad0, pad1, pad2;
    uint32_t rank;
    uint32_t pad3;
};
static_assert(sizeof(Lane) == 64, "lane layout");

struct Tables {               // each 4097 int64
    const int64_t* kern;      // lognormal kernel durations
    const int64_t* copy;      // lognormal copy durations
    const int64_t* expo;      // exponential, mean 1e6
};

__device__ __forceinline__ uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t j, uint32_t t) {
    return mix(key ^ ((j << 3 | t) * 0xD6E8FEB86659FD93ull));
}

__device__ __forceinline__ int64_t tab(const int64_t* T, uint64_t u) {
    const uint32_t i = static_cast<uint32_t>(u >> 52);
    const int64_t f = static_cast<int64_t>((u >> 36) & 0xFFFFull);
    return T[i] + (((T[i + 1] - T[i]) * f) >> 16);
}

struct Slot {
    int64_t len;   // kernel + gap (device) or interval (host)
    int64_t kd;    // kernel duration (device) / state (host)
    int64_t gap;
};

__device__ __forceinline__ Slot slot_of(const Lane& L, const Tables& tb, uint64_t j) {
    Slot s;
    if (L.is_host) {
        const uint64_t u0 = draw(L.key, j, 0);
        const uint32_t state = static_cast<uint32_t>((u0 >> 32) % 3u);
        const int64_t mean = state == 0 ? 50000 : (state == 1 ? 5000 : 10000);
        s.len = tab(tb.expo, draw(L.key, j, 1)) * mean / 1000000;
        s.kd = state;
        s.gap = 0;
    } else {
        const uint64_t u0 = draw(L.key, j, 0);
        int64_t kd;
        if (L.law == 0) kd = tab(tb.kern, u0);
        else kd = (u0 >> 11) < 7205759403792794ull ? 1000 : 500000;   // 0.8 * 2^53
        kd = kd * static_cast<int64_t>(L.work_milli) / 1000;
        if (kd < 1) kd = 1;
        const int64_t gap = tab(tb.expo, draw(L.key, j, 1)) * L.mean_gap / 1000000;
        s.len = kd + gap;
        s.kd = kd;
        s.gap = gap;
    }
    return s;
}

__device__ __forceinline__ uint64_t lane_slots(const Lane& L) {
    return L.is_host ? L.n : (7 * L.n + 5) / 10;
}

template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int m = 16; m > 0; m >>= 1) v = op(v, __shfl_xor_sync(0xFFFFFFFFu, v, m));
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T r = sh[0];
    for (int i = 1; i < kThreads / 32; ++i) r = op(r, sh[i]);
    __syncthreads();
    return r;
}

// exclusive block scan of one int64 per thread
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= d) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    int64_t base = 0;
    for (int i = 0; i < wid; ++i) base += sh[i];
    __syncthreads();
    return base + x - v;
}

__global__ void __launch_bounds__(kThreads) chunk_sums(const Lane* __restrict__ lanes,
                                                       const uint32_t* __restrict__ chunk_lane, Tables tb,
                                                       int64_t* __restrict__ sums) {
    __shared__ int64_t sh[32];
    const uint32_t c = blockIdx.x;
    const Lane L = lanes[chunk_lane[c]];
    const uint64_t S = lane_slots(L);
    const uint64_t j0 = static_cast<uint64_t>(c - L.chunk0) * kChunk + threadIdx.x * kPer;
    int64_t acc = 0;
    for (int k = 0; k < kPer; ++k) {
        const uint64_t j = j0 + k;
        if (j < S) acc += slot_of(L, tb, j).len;
    }
    acc = block_reduce<int64_t>(acc, [](int64_t a, int64_t b) { return a + b; }, sh);
    if (threadIdx.x == 0) sums[c] = acc;
}

// one warp per lane: exclusive prefix of its chunk sums, from t0
__global__ void chunk_scan(const Lane* __restrict__ lanes, uint32_t n_lanes, const int64_t* __restrict__ sums,
                           int64_t* __restrict__ base) {
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_lanes) return;
    const Lane L = lanes[w];
    const uint64_t S = lane_slots(L);
    const uint32_t nc = static_cast<uint32_t>((S + kChunk - 1) / kChunk);
    int64_t run = L.t0;
    for (uint32_t c0 = 0; c0 < nc; c0 += 32) {
        const uint32_t c = c0 + lane;
        const int64_t v = c < nc ? sums[L.chunk0 + c] : 0;
        int64_t x = v;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if (lane >= d) x += y;
        }
        if (c < nc) base[L.chunk0 + c] = run + x - v;
        run += __shfl_sync(0xFFFFFFFFu, x, 31);
    }
}

__global__ void __launch_bounds__(kThreads) write_rows(const Lane* __restrict__ lanes,
                                                       const uint32_t* __restrict__ chunk_lane, Tables tb,
                                                       const int64_t* __restrict__ base, int64_t* __restrict__ dse,
                                                       uint8_t* __restrict__ dtag, int64_t* __restrict__ hse,
                                                       uint8_t* __restrict__ hstate,
                                                       unsigned long long* __restrict__ lane_end) {
    __shared__ int64_t sh[32];
    const uint32_t c = blockIdx.x;
    const uint32_t li = chunk_lane[c];
    const Lane L = lanes[li];
    const uint64_t S = lane_slots(L);
    const uint64_t C = L.is_host ? 0 : L.n - S;
    const uint64_t j0 = static_cast<uint64_t>(c - L.chunk0) * kChunk + threadIdx.x * kPer;
    Slot sl[kPer];
    int64_t tot = 0;
    for (int k = 0; k < kPer; ++k) {
        const uint64_t j = j0 + k;
        if (j < S) {
            sl[k] = slot_of(L, tb, j);
            tot += sl[k].len;
        } else {
            sl[k].len = sl[k].kd = sl[k].gap = 0;
        }
    }
    int64_t t = base[c] + block_excl_scan(tot, sh);
    int64_t mx = INT64_MIN;
    for (int k = 0; k < kPer; ++k) {
        const uint64_t j = j0 + k;
        if (j >= S) break;
        if (L.is_host) {
            const uint64_t r = L.out + j;
            hse[2 * r] = t;
            hse[2 * r + 1] = t + sl[k].len;
            hstate[r] = static_cast<uint8_t>(sl[k].kd);
            mx = max(mx, t + sl[k].len);
        } else {
            const int64_t kd = sl[k].kd, gap = sl[k].gap;
            const uint64_t e = j + (j * C) / S;
            const uint64_t r = L.out + e;
            dse[2 * r] = t;
            dse[2 * r + 1] = t + kd;
            dtag[r] = static_cast<uint8_t>(j % L.n_kstreams);
            mx = max(mx, t + kd);
            const bool has = ((j + 1) * C) / S - (j * C) / S != 0;
            if (has) {
                const bool inside = (draw(L.key, j, 2) >> 32) < 1288490189ull;   // 0.3 * 2^32
                const int64_t f = static_cast<int64_t>(draw(L.key, j, 3) >> 40);
                const int64_t cs = inside ? t + ((kd * f) >> 24) : t + kd + ((gap * f) >> 24);
                int64_t cd = tab(tb.copy, draw(L.key, j, 4));
                if (cd < 1) cd = 1;
                const uint32_t kind = 1u + static_cast<uint32_t>(draw(L.key, j, 5) & 1u);
                dse[2 * (r + 1)] = cs;
                dse[2 * (r + 1) + 1] = cs + cd;
                dtag[r + 1] = static_cast<uint8_t>(kind << 5 | (L.copy_stream0 + j % L.n_cstreams));
                mx = max(mx, cs + cd);
            }
        }
        t += sl[k].len;
    }
    mx = block_reduce<int64_t>(mx, [](int64_t a, int64_t b) { return a > b ? a : b; }, sh);
    // ends are >= 0 here, so an unsigned max orders them correctly
    if (threadIdx.x == 0 && mx != INT64_MIN) atomicMax(&lane_end[li], static_cast<unsigned long long>(mx));
}

// per rank: T = max(host end, its devices' last ends, 1); the pad interval
// [host end, T) closes the host lane
__global__ void pad_ranks(const Lane* __restrict__ lanes, const uint32_t* __restrict__ rank_host,
                          const uint32_t* __restrict__ rank_dev0, const uint32_t* __restrict__ rank_ndev,
                          uint32_t n_ranks, const unsigned long long* __restrict__ lane_end,
                          int64_t* __restrict__ hse, uint8_t* __restrict__ hstate, int64_t* __restrict__ T_out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_ranks) return;
    const Lane H = lanes[rank_host[i]];
    const int64_t hend = H.n ? static_cast<int64_t>(lane_end[rank_host[i]]) : H.t0;
    int64_t T = hend > 1 ? hend : 1;
    for (uint32_t k = 0; k < rank_ndev[i]; ++k) {
        const uint32_t g = rank_dev0[i] + k;
        if (lanes[g].n) T = max(T, static_cast<int64_t>(lane_end[g]));
    }
    const uint64_t r = H.out + H.n;
    hse[2 * r] = hend;
    hse[2 * r + 1] = T > hend ? T : hend;
    hstate[r] = 1;
    T_out[i] = T;
}

}  // namespace

extern "C" {

// Generate every lane of `lanes` (device memory, n_lanes entries; device
// lanes first is not required).  chunk_lane[n_chunks] maps each chunk of
// kChunk slots to its lane; rank_* describe each rank's host lane and its
// contiguous device lanes.  Scratch: sums/base [n_chunks] int64, lane_end
// [n_lanes] u64 (zeroed here).  Returns a cudaError_t code.
int igen_generate(const void* lanes, uint32_t n_lanes, const uint32_t* chunk_lane, uint32_t n_chunks,
                  const int64_t* tab_kern, const int64_t* tab_copy, const int64_t* tab_expo, int64_t* sums,
                  int64_t* base, unsigned long long* lane_end, int64_t* dse, uint8_t* dtag, int64_t* hse,
                  uint8_t* hstate, const uint32_t* rank_host, const uint32_t* rank_dev0, const uint32_t* rank_ndev,
                  uint32_t n_ranks, int64_t* T_out, void* stream_) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    const Lane* L = static_cast<const Lane*>(lanes);
    Tables tb{tab_kern, tab_copy, tab_expo};
    cudaError_t e = cudaMemsetAsync(lane_end, 0, sizeof(unsigned long long) * n_lanes, stream);
    if (e != cudaSuccess) return e;
    if (n_chunks) {
        chunk_sums<<<n_chunks, kThreads, 0, stream>>>(L, chunk_lane, tb, sums);
        chunk_scan<<<(n_lanes + 7) / 8, 256, 0, stream>>>(L, n_lanes, sums, base);
        write_rows<<<n_chunks, kThreads, 0, stream>>>(L, chunk_lane, tb, base, dse, dtag, hse, hstate, lane_end);
    }
    if (n_ranks)
        pad_ranks<<<(n_ranks + 255) / 256, 256, 0, stream>>>(L, rank_host, rank_dev0, rank_ndev, n_ranks, lane_end,
                                                            hse, hstate, T_out);
    return static_cast<int>(cudaGetLastError());
}

int igen_chunk_slots(void) { return kChunk; }

}  // extern "C"
