// Per-lane arithmetic of the sweep (Sec. 4.2 flattening and the Sec. 4.1
// host-state sums), shared by the streaming sweep (records already in start
// order) and the fused merge-sweep (records merged from sorted runs in
// shared memory).  Records are held in registers as 32-bit offsets from a
// base start s0; 0 stands for "no earlier record".
#pragma once
#include "common.cuh"

namespace talp {

__device__ __forceinline__ uint32_t umax(uint32_t a, uint32_t b) { return a > b ? a : b; }
__device__ __forceinline__ uint32_t umin(uint32_t a, uint32_t b) { return a < b ? a : b; }

// Warp sum of per-lane values below 2^51 with two hardware 32-bit reductions.
__device__ __forceinline__ int64_t warp_sum_u64_small(uint64_t v) {
    const uint32_t lo = __reduce_add_sync(0xFFFFFFFFu, static_cast<uint32_t>(v & 0xFFFFFull));
    const uint32_t hi = __reduce_add_sync(0xFFFFFFFFu, static_cast<uint32_t>(v >> 20));
    return static_cast<int64_t>((static_cast<uint64_t>(hi) << 20) + lo);
}

// a window bound relative to s0, saturated to [0, 2^32 - 1]
__device__ __forceinline__ uint32_t rel_sat(int64_t x, int64_t s0) {
    if (x <= s0) return 0u;
    const uint64_t d = static_cast<uint64_t>(x - s0);
    return d > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(d);
}

// Validation and lane aggregates of a device tile (32-bit offsets): all ends
// >= starts, kinds <= 4 (tag < 160), starts non-decreasing; largest kernel
// and memory end of the lane (0 = none).  A tag below 32 is a kernel.
template <int ITEMS, bool FULL>
__device__ __forceinline__ void dev_pass1(const uint32_t (&sr)[ITEMS], const uint32_t (&er)[ITEMS],
                                          const uint32_t (&tg)[ITEMS], int cnt, uint32_t& aK, uint32_t& aM,
                                          bool& okE, bool& okS, bool& okK) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (FULL || i < cnt) {
            const uint32_t t = tg[i];
            okE = okE & (er[i] >= sr[i]);
            okK = okK & (t < 160u);
            if (i > 0) okS = okS & (sr[i] >= sr[i - 1]);
            const bool isK = t < 32u;
            aK = isK ? umax(aK, er[i]) : aK;
            aM = isK ? aM : umax(aM, er[i]);
        }
    }
}

// New pieces of one lane's records (32-bit offsets), clipped to [a, b)
// (a = 0, b = 2^32 - 1: unclipped).  Kp/Mp: largest kernel / memory end
// before the lane's first record.  sK, sM, sA must enter as 0.
template <int ITEMS, bool FULL>
__device__ __forceinline__ void pieces32(const uint32_t (&sr)[ITEMS], const uint32_t (&er)[ITEMS],
                                         const uint32_t (&tg)[ITEMS], int cnt, uint32_t Kp, uint32_t Mp,
                                         uint32_t a, uint32_t b, uint32_t& sK, uint32_t& sM, uint32_t& sA) {
    uint32_t Ap = umax(Kp, Mp), sO = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (FULL || i < cnt) {
            const bool isK = tg[i] < 32u;
            const uint32_t own = isK ? Kp : Mp;
            const uint32_t pA = umax(umax(sr[i], Ap), a);
            const uint32_t pO = umax(umax(sr[i], own), a);
            const uint32_t e = umin(er[i], b);
            sA += umax(e, pA) - pA;
            const uint32_t lO = umax(e, pO) - pO;
            sO += lO;
            sK += isK ? lO : 0u;
            const uint32_t nw = umax(own, er[i]);
            Kp = isK ? nw : Kp;
            Mp = isK ? Mp : nw;
            Ap = umax(Ap, er[i]);
        }
    }
    sM += sO - sK;
}

// The start of each record's new piece in the all-records chain (written
// over sr) and in its own chain (pO), with the lane's carries Kp / Mp: the
// part of pieces32 that does not depend on the window, for tiles clipped to
// several windows.
template <int ITEMS>
__device__ __forceinline__ void piece_starts(uint32_t (&sr)[ITEMS], uint32_t (&pO)[ITEMS],
                                             const uint32_t (&er)[ITEMS], const uint32_t (&tg)[ITEMS], int cnt,
                                             uint32_t Kp, uint32_t Mp) {
    uint32_t Ap = umax(Kp, Mp);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        pO[i] = 0;
        if (i < cnt) {
            const bool isK = tg[i] < 32u;
            const uint32_t own = isK ? Kp : Mp;
            pO[i] = umax(sr[i], own);
            sr[i] = umax(sr[i], Ap);
            const uint32_t nw = umax(own, er[i]);
            Kp = isK ? nw : Kp;
            Mp = isK ? Mp : nw;
            Ap = umax(Ap, er[i]);
        }
    }
}

// pieces32 clipped to [a, b) from the piece starts (pA, pO) of piece_starts:
// the same sums.
template <int ITEMS>
__device__ __forceinline__ void clip_pieces(const uint32_t (&pA)[ITEMS], const uint32_t (&pO)[ITEMS],
                                            const uint32_t (&er)[ITEMS], const uint32_t (&tg)[ITEMS], int cnt,
                                            uint32_t a, uint32_t b, uint32_t& sK, uint32_t& sM, uint32_t& sA) {
    uint32_t sO = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (i < cnt) {
            const uint32_t e = umin(er[i], b);
            const uint32_t pa = umax(pA[i], a);
            sA += umax(e, pa) - pa;
            const uint32_t po = umax(pO[i], a);
            const uint32_t lO = umax(e, po) - po;
            sO += lO;
            sK += tg[i] < 32u ? lO : 0u;
        }
    }
    sM += sO - sK;
}

// Host tile (32-bit offsets): per-state sums of lengths clipped to [a, b),
// the lane's smallest start and largest end, and validation.
template <int ITEMS, bool FULL>
__device__ __forceinline__ void host_pass(const uint32_t (&sr)[ITEMS], const uint32_t (&er)[ITEMS],
                                          const uint32_t (&tg)[ITEMS], int cnt, uint32_t a, uint32_t b,
                                          uint64_t& h0, uint64_t& h1, uint64_t& h2, uint32_t& lo, uint32_t& hi,
                                          bool& okE, bool& okK) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (FULL || i < cnt) {
            const uint32_t q = tg[i];
            okE = okE & (er[i] >= sr[i]);
            okK = okK & (q < 3u);
            const uint32_t p = umax(sr[i], a);
            const uint64_t l = umax(umin(er[i], b), p) - p;
            h0 += q == 0u ? l : 0ull;
            h1 += q == 1u ? l : 0ull;
            h2 += q == 2u ? l : 0ull;
            lo = umin(lo, sr[i]);
            hi = umax(hi, er[i]);
        }
    }
}

// Same in absolute int64 from the shared-memory tile (the exact path).
template <int ITEMS>
__device__ __forceinline__ void pieces64(const longlong2* sse, int base, const uint32_t (&tg)[ITEMS], int cnt,
                                         int64_t Kp, int64_t Mp, int64_t a, int64_t b, int64_t& sK, int64_t& sM,
                                         int64_t& sA) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (i < cnt) {
            const longlong2 v = sse[base + i];
            const bool isK = (tg[i] >> 5) == 0u;
            const int64_t pA = max64(max64(v.x, max64(Kp, Mp)), a);
            const int64_t pO = max64(max64(v.x, isK ? Kp : Mp), a);
            const int64_t e = min64(v.y, b);
            sA += max64(e - pA, 0);
            const int64_t lO = max64(e - pO, 0);
            if (isK) {
                sK += lO;
                Kp = max64(Kp, v.y);
            } else {
                sM += lO;
                Mp = max64(Mp, v.y);
            }
        }
    }
}

}  // namespace talp
