// Sweep kernel: the flattening of Sec. 4.2 and the host-state sums of
// Sec. 4.1 in one persistent pass over every record of the ingest.
//
// Device segment (one GPU of one rank, records in start order).  With the
// records sorted by start, the part of record j not covered by any earlier
// record of a set X is [max(s_j, P_X(j)), e_j), P_X(j) being the largest end
// of the earlier records of X.  These "new pieces" are disjoint, so
//   |union of X, clipped to [a, b)| = sum_j |[max(s_j, P_X(j), a), min(e_j, b))|.
// Three chains are kept per device: X = kernels (D_K), X = memory
// operations (their union) and X = all records (busy time B); the transfer
// time not hidden by kernels is D_M = B - D_K (Sec. 4.1: overlap counts as
// computation; Sec. 4.2: transfer parts under kernels removed).
//
// Host segment (one rank): per state, the plain sum of clipped lengths
// (Eq. 2 for useful, offload and MPI time).
//
// Work split: the ingest's records form one virtual array (segments back to
// back).  Each warp of the persistent grid owns an equal contiguous slice and
// streams it in tiles of 32*ITEMS records through its own STAGES-deep ring of
// shared-memory buffers filled by 1-D bulk TMA copies (cp.async.bulk) that
// complete on per-stage mbarriers.  No CTA-wide barrier exists: warps are
// independent.  Lane l holds records [l*ITEMS, (l+1)*ITEMS) of a tile
// (blocked), so each lane scans its records serially and the warp combines
// lane aggregates with one shuffle max-scan per tile.
//
// A warp whose slice starts inside a device segment does not know the
// running max end of the records before its slice; it starts that chain
// empty and the fix-up kernel later subtracts the over-count (the part of the
// slice's new pieces that lies below the true carry), which only touches the
// few records whose start lies below the carry.  No warp ever waits on
// another.
//
// Each lane classifies its records of a tile against each region window by
// their span [first start, max end]: fully inside adds the unclipped piece
// sums, fully outside adds nothing, and only a straddling lane recomputes its
// pieces clipped.
#include "kernels.h"

namespace talp {

const SweepShape kSweepShapes[kNumSweepShapes] = {
    {7, 8, 4},   // 224-record tiles, 8 warps, 4 stages
    {9, 8, 3},   // 288-record tiles, 8 warps, 3 stages
    {7, 4, 6},   // 224-record tiles, 4 warps, 6 stages
    {5, 8, 4},   // 160-record tiles, 8 warps, 4 stages
};

template <int ITEMS, int WARPS, int STAGES, int RMAX>
struct SweepCfg {
    static constexpr int TILE = 32 * ITEMS;
    static constexpr int SE_BYTES = TILE * 16;
    static constexpr int TAG_BYTES = TILE + 32;                 // 16-byte aligned superset of a tile's tags
    static constexpr int STAGE_BYTES = SE_BYTES + TAG_BYTES;    // multiple of 16
    static constexpr int WIN_BYTES = RMAX * 16;
    static constexpr int RAW = STAGES * STAGE_BYTES + STAGES * 8 + WIN_BYTES;
    static constexpr int WARP_BYTES = (RAW + 127) / 128 * 128;
    static constexpr int SMEM = WARPS * WARP_BYTES;
};

// Position of a warp inside its slice: current tile start, current segment,
// end of the current portion (segment end or slice end).
struct Walk {
    uint64_t pos, seg_end, seg_base;
    uint32_t seg;
};

__device__ __forceinline__ void walk_enter(Walk& w, const uint64_t* __restrict__ seg_start, uint64_t r1) {
    while (seg_start[w.seg + 1] <= w.pos) ++w.seg;   // skip empty segments
    w.seg_base = seg_start[w.seg];
    const uint64_t e = seg_start[w.seg + 1];
    w.seg_end = e < r1 ? e : r1;
}

// Returns true when the walk moved into a new segment.
__device__ __forceinline__ bool walk_advance(Walk& w, uint32_t len, const uint64_t* __restrict__ seg_start,
                                             uint64_t r1) {
    w.pos += len;
    if (w.pos < r1 && w.pos == w.seg_end) {
        ++w.seg;
        walk_enter(w, seg_start, r1);
        return true;
    }
    return false;
}

template <int ITEMS, int WARPS, int STAGES, int RMAX>
__global__ void __launch_bounds__(WARPS * 32)
    sweep_kernel(const SegDesc* __restrict__ segs, const uint64_t* __restrict__ seg_start, uint32_t n_segs,
                 WarpRec* __restrict__ wrec, uint32_t* __restrict__ seg_flags, uint32_t* __restrict__ gstatus,
                 int64_t wait_limit) {
    using C = SweepCfg<ITEMS, WARPS, STAGES, RMAX>;
    constexpr int TILE = C::TILE;
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    uint8_t* wsm = smem + wid * C::WARP_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wsm + STAGES * C::STAGE_BYTES);
    int64_t* swin = reinterpret_cast<int64_t*>(wsm + STAGES * C::STAGE_BYTES + STAGES * 8);

    const uint64_t GW = static_cast<uint64_t>(gridDim.x) * WARPS;
    const uint64_t gw = static_cast<uint64_t>(blockIdx.x) * WARPS + wid;
    const uint64_t N = seg_start[n_segs];
    const uint64_t r0 = (N * gw) / GW;
    const uint64_t r1 = (N * (gw + 1)) / GW;

    if (r0 >= r1) {
        if (lane == 0) {
            WarpRec rec;
            rec.head_pos = r0;
            rec.head_end = r0;
            rec.head_seg = NONE;
            rec.tail_seg = NONE;
            rec.head_K = rec.head_M = rec.tail_K = rec.tail_M = NEG_INF;
            wrec[gw] = rec;
        }
        return;
    }

    // segment containing r0: the last index whose start is <= r0
    uint32_t lo = 0, hi = n_segs;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (seg_start[mid] <= r0) lo = mid; else hi = mid;
    }

    if (lane == 0) {
#pragma unroll
        for (int st = 0; st < STAGES; ++st) mbar_init(&bars[st], 1);
        fence_mbar_init();
    }
    __syncwarp();

    // ---- producer (lane 0): its own walk over the same tile sequence
    Walk iw;
    iw.pos = r0;
    iw.seg = lo;
    walk_enter(iw, seg_start, r1);
    uint32_t n_issued = 0;
    bool iw_done = false;

    auto issue = [&](int st) {
        const SegDesc& d = segs[iw.seg];
        const uint64_t off = iw.pos - iw.seg_base;
        const uint64_t rem = iw.seg_end - iw.pos;
        const uint32_t len = rem < static_cast<uint64_t>(TILE) ? static_cast<uint32_t>(rem) : TILE;
        uint8_t* stage = wsm + st * C::STAGE_BYTES;
        const uintptr_t A = reinterpret_cast<uintptr_t>(d.tag + off);
        const uintptr_t tlo = A & ~static_cast<uintptr_t>(15);
        uintptr_t thi = (A + len + 15) & ~static_cast<uintptr_t>(15);
        const uintptr_t lim = reinterpret_cast<uintptr_t>(d.tag_limit);
        if (thi > lim) thi = lim;
        const uint32_t tag_bytes = thi > tlo ? static_cast<uint32_t>(thi - tlo) : 0u;
        mbar_arrive_expect_tx(&bars[st], len * 16u + tag_bytes);
        tma_load_1d(stage, d.se + 2 * off, len * 16u, &bars[st]);
        if (tag_bytes) tma_load_1d(stage + C::SE_BYTES, reinterpret_cast<const void*>(tlo), tag_bytes, &bars[st]);
        ++n_issued;
        if (iw.pos + len >= r1) {
            iw_done = true;
        } else {
            walk_advance(iw, len, seg_start, r1);
        }
    };

    if (lane == 0) {
        for (int st = 0; st < STAGES && !iw_done; ++st) issue(st);
    }

    // ---- consumers (all lanes): the same walk
    Walk cw;
    cw.pos = r0;
    cw.seg = lo;
    walk_enter(cw, seg_start, r1);

    WarpRec rec;
    rec.head_pos = r0;
    rec.head_seg = cw.seg;
    rec.head_end = cw.seg_end;
    rec.head_K = rec.head_M = NEG_INF;
    rec.tail_seg = NONE;
    rec.tail_K = rec.tail_M = NEG_INF;
    bool first_portion = true;

    int64_t acc[RMAX][3];
    int64_t carryK = NEG_INF, carryM = NEG_INF, last_s = NEG_INF;
    uint32_t pbad = 0;
    SegDesc d;
    bool portion_open = false;
    uint32_t n_consumed = 0;
    bool timed_out = false;

    while (true) {
        if (!portion_open) {
            d = segs[cw.seg];
#pragma unroll
            for (int r = 0; r < RMAX; ++r) acc[r][0] = acc[r][1] = acc[r][2] = 0;
            pbad = 0;
            if (!d.is_host && cw.pos == cw.seg_base) {
                carryK = d.carry_in[0];
                carryM = d.carry_in[1];
                last_s = d.carry_in[2];
            } else {
                carryK = carryM = last_s = NEG_INF;
            }
            if (lane < 2 * RMAX && lane < 2 * d.R) swin[lane] = d.win[lane];
            __syncwarp();
            portion_open = true;
        }
        const int st = static_cast<int>(n_consumed % STAGES);
        const uint32_t ph = (n_consumed / STAGES) & 1u;
        const bool ok = mbar_wait_bounded(&bars[st], ph, wait_limit);
        if (__any_sync(0xFFFFFFFFu, !ok)) {
            timed_out = true;
            break;
        }
        const uint8_t* stage = wsm + st * C::STAGE_BYTES;
        const longlong2* sse = reinterpret_cast<const longlong2*>(stage);
        const uint64_t off = cw.pos - cw.seg_base;
        const uint64_t rem = cw.seg_end - cw.pos;
        const int len = rem < static_cast<uint64_t>(TILE) ? static_cast<int>(rem) : TILE;
        const uintptr_t A = reinterpret_cast<uintptr_t>(d.tag + off);
        const int toff = static_cast<int>(A & 15u);
        const uintptr_t lim = reinterpret_cast<uintptr_t>(d.tag_limit);
        const int direct_from = lim > A ? static_cast<int>(min(static_cast<uint64_t>(lim - A), static_cast<uint64_t>(len))) : 0;
        const uint8_t* stag = stage + C::SE_BYTES + toff;
        const uint8_t* gtag = d.tag + off;

        const int base = lane * ITEMS;
        const int cnt = max(0, min(ITEMS, len - base));
        int64_t s_[ITEMS], e_[ITEMS];
        uint32_t t_[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if (i < cnt) {
                const longlong2 v = sse[base + i];
                s_[i] = v.x;
                e_[i] = v.y;
                const int k = base + i;
                t_[i] = k < direct_from ? stag[k] : __ldg(gtag + k);
            } else {
                s_[i] = 0;
                e_[i] = 0;
                t_[i] = 0;
            }
        }
        const int64_t prev_s = (cnt > 0) ? (lane == 0 ? last_s : sse[base - 1].x) : 0;
        const int64_t tile_last_s = sse[len - 1].x;
        __syncwarp();
        if (lane == 0) {
            fence_proxy_async_smem();
            if (!iw_done) issue(st);
        }
        ++n_consumed;

        uint32_t bad = 0;
        if (!d.is_host) {
            // pass 1: validation and lane aggregates of the kernel / memory ends
            int64_t aK = NEG_INF, aM = NEG_INF;
            int64_t ps = prev_s;
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (i < cnt) {
                    const uint32_t kind = t_[i] >> 5;
                    bad |= (e_[i] < s_[i]) ? ST_BAD_END : 0u;
                    bad |= (kind > 4u) ? ST_BAD_KIND : 0u;
                    bad |= (s_[i] < ps) ? ST_UNSORTED : 0u;
                    ps = s_[i];
                    if (kind == 0u) aK = max64(aK, e_[i]); else aM = max64(aM, e_[i]);
                }
            }
            // warp exclusive max-scan of the lane aggregates, seeded by the carry
            int64_t iK = aK, iM = aM;
            warp_incl_max2(iK, iM, lane);
            int64_t xK = shfl_up64(iK, 1), xM = shfl_up64(iM, 1);
            if (lane == 0) {
                xK = NEG_INF;
                xM = NEG_INF;
            }
            xK = max64(xK, carryK);
            xM = max64(xM, carryM);
            carryK = max64(carryK, shfl64(iK, 31));
            carryM = max64(carryM, shfl64(iM, 31));

            if (cnt > 0) {
                // pass 2: unclipped new pieces of the three chains
                int64_t sK = 0, sM = 0, sA = 0;
                {
                    int64_t Kp = xK, Mp = xM;
#pragma unroll
                    for (int i = 0; i < ITEMS; ++i) {
                        if (i < cnt) {
                            const bool isK = (t_[i] >> 5) == 0u;
                            const int64_t pA = max64(s_[i], max64(Kp, Mp));
                            const int64_t pO = max64(s_[i], isK ? Kp : Mp);
                            sA += max64(e_[i] - pA, 0);
                            const int64_t lO = max64(e_[i] - pO, 0);
                            if (isK) {
                                sK += lO;
                                Kp = max64(Kp, e_[i]);
                            } else {
                                sM += lO;
                                Mp = max64(Mp, e_[i]);
                            }
                        }
                    }
                }
                const int64_t lo_t = s_[0];
                const int64_t hi_t = max64(aK, aM);
#pragma unroll
                for (int r = 0; r < RMAX; ++r) {
                    if (r < d.R) {
                        const int64_t a = swin[2 * r], b = swin[2 * r + 1];
                        if (lo_t >= a && hi_t <= b) {
                            acc[r][0] += sK;
                            acc[r][1] += sM;
                            acc[r][2] += sA;
                        } else if (!(hi_t <= a || lo_t >= b)) {
                            int64_t Kp = xK, Mp = xM, cK = 0, cM = 0, cA = 0;
#pragma unroll
                            for (int i = 0; i < ITEMS; ++i) {
                                if (i < cnt) {
                                    const bool isK = (t_[i] >> 5) == 0u;
                                    const int64_t pA = max64(s_[i], max64(Kp, Mp));
                                    const int64_t pO = max64(s_[i], isK ? Kp : Mp);
                                    const int64_t eb = min64(e_[i], b);
                                    cA += max64(eb - max64(pA, a), 0);
                                    const int64_t lO = max64(eb - max64(pO, a), 0);
                                    if (isK) {
                                        cK += lO;
                                        Kp = max64(Kp, e_[i]);
                                    } else {
                                        cM += lO;
                                        Mp = max64(Mp, e_[i]);
                                    }
                                }
                            }
                            acc[r][0] += cK;
                            acc[r][1] += cM;
                            acc[r][2] += cA;
                        }
                    }
                }
            }
        } else {
            // host: per-state sums of clipped lengths
            int64_t u = 0, w = 0, p = 0;
            int64_t lo_t = INT64_MAX, hi_t = NEG_INF;
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (i < cnt) {
                    const uint32_t q = t_[i];
                    bad |= (e_[i] < s_[i]) ? ST_BAD_END : 0u;
                    bad |= (q > 2u) ? ST_BAD_KIND : 0u;
                    const int64_t l = max64(e_[i] - s_[i], 0);
                    u += (q == 0u) ? l : 0;
                    w += (q == 1u) ? l : 0;
                    p += (q == 2u) ? l : 0;
                    lo_t = min64(lo_t, s_[i]);
                    hi_t = max64(hi_t, e_[i]);
                }
            }
            if (cnt > 0) {
#pragma unroll
                for (int r = 0; r < RMAX; ++r) {
                    if (r < d.R) {
                        const int64_t a = swin[2 * r], b = swin[2 * r + 1];
                        if (lo_t >= a && hi_t <= b) {
                            acc[r][0] += u;
                            acc[r][1] += w;
                            acc[r][2] += p;
                        } else if (!(hi_t <= a || lo_t >= b)) {
                            int64_t cu = 0, cw2 = 0, cp = 0;
#pragma unroll
                            for (int i = 0; i < ITEMS; ++i) {
                                if (i < cnt) {
                                    const uint32_t q = t_[i];
                                    const int64_t l = max64(min64(e_[i], b) - max64(s_[i], a), 0);
                                    cu += (q == 0u) ? l : 0;
                                    cw2 += (q == 1u) ? l : 0;
                                    cp += (q == 2u) ? l : 0;
                                }
                            }
                            acc[r][0] += cu;
                            acc[r][1] += cw2;
                            acc[r][2] += cp;
                        }
                    }
                }
            }
        }
        pbad |= bad;
        last_s = tile_last_s;

        // advance; close the portion when the segment (or the slice) ends
        const bool slice_done = cw.pos + static_cast<uint64_t>(len) >= r1;
        const bool seg_done = slice_done || (cw.pos + static_cast<uint64_t>(len) == cw.seg_end);
        if (seg_done) {
#pragma unroll
            for (int r = 0; r < RMAX; ++r) {
                if (r < d.R) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const int64_t v = warp_sum64(acc[r][c]);
                        if (lane == 0 && v != 0) atomic_add64(&d.sums[3 * r + c], v);
                    }
                }
            }
            const uint32_t bits = __reduce_or_sync(0xFFFFFFFFu, pbad);
            if (lane == 0) {
                if (bits) {
                    atomicOr(d.status, bits);
                    atomicOr(&seg_flags[cw.seg], bits);
                }
                if (!d.is_host) {
                    atomic_max64(&d.carry_out[0], carryK);
                    atomic_max64(&d.carry_out[1], carryM);
                    atomic_max64(&d.carry_out[2], last_s);
                }
            }
            if (first_portion) {
                rec.head_K = carryK;
                rec.head_M = carryM;
                first_portion = false;
            }
            rec.tail_seg = cw.seg;
            rec.tail_K = carryK;
            rec.tail_M = carryM;
            portion_open = false;
        }
        if (slice_done) break;
        walk_advance(cw, static_cast<uint32_t>(len), seg_start, r1);
    }

    if (timed_out) {
        if (lane == 0) {
            atomicOr(gstatus, ST_TIMEOUT);
            atomicOr(d.status, ST_TIMEOUT);
            // let the copies still in flight land before the CTA's shared memory goes away
            for (uint32_t t = n_consumed; t < n_issued; ++t)
                (void)mbar_wait_bounded(&bars[t % STAGES], (t / STAGES) & 1u, wait_limit);
            rec.head_seg = NONE;
            rec.tail_seg = NONE;
            wrec[gw] = rec;
        }
        return;
    }
    if (lane == 0) wrec[gw] = rec;
}

// ---------------------------------------------------------------- dispatch

template <int ITEMS, int WARPS, int STAGES, int RMAX>
static cudaError_t launch_t(int grid, const SegDesc* segs, const uint64_t* seg_start, uint32_t n_segs,
                            WarpRec* wrec, uint32_t* seg_flags,
                            uint32_t* gstatus, int64_t wait_limit, cudaStream_t stream) {
    using C = SweepCfg<ITEMS, WARPS, STAGES, RMAX>;
    auto k = sweep_kernel<ITEMS, WARPS, STAGES, RMAX>;
    static bool attr_set = false;   // per-instantiation, set once per process
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k<<<grid, WARPS * 32, C::SMEM, stream>>>(segs, seg_start, n_segs, wrec, seg_flags, gstatus, wait_limit);
    return cudaGetLastError();
}

template <int ITEMS, int WARPS, int STAGES, int RMAX>
static int occupancy_t() {
    using C = SweepCfg<ITEMS, WARPS, STAGES, RMAX>;
    auto k = sweep_kernel<ITEMS, WARPS, STAGES, RMAX>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, WARPS * 32, C::SMEM) != cudaSuccess) return 0;
    return n;
}

#define TALP_SHAPE_SWITCH(shape, RM, CALL)                \
    switch (shape) {                                      \
        case 0: return CALL(7, 8, 4, RM);                 \
        case 1: return CALL(9, 8, 3, RM);                 \
        case 2: return CALL(7, 4, 6, RM);                 \
        case 3: return CALL(5, 8, 4, RM);                 \
        default: break;                                   \
    }

#define TALP_LAUNCH(I, W, S, RM) \
    launch_t<I, W, S, RM>(grid, segs, seg_start, n_segs, wrec, seg_flags, gstatus, wait_limit, stream)
#define TALP_OCC(I, W, S, RM) occupancy_t<I, W, S, RM>()

cudaError_t launch_sweep(int shape, int rmax, int grid, const SegDesc* segs, const uint64_t* seg_start,
                         uint32_t n_segs, WarpRec* wrec, uint32_t* seg_flags, uint32_t* gstatus, int64_t wait_limit,
                         cudaStream_t stream) {
    if (rmax <= 1) { TALP_SHAPE_SWITCH(shape, 1, TALP_LAUNCH) }
    else if (rmax <= 2) { TALP_SHAPE_SWITCH(shape, 2, TALP_LAUNCH) }
    else if (rmax <= 4) { TALP_SHAPE_SWITCH(shape, 4, TALP_LAUNCH) }
    else { TALP_SHAPE_SWITCH(shape, 8, TALP_LAUNCH) }
    return cudaErrorInvalidValue;
}

int sweep_ctas_per_sm(int shape, int rmax) {
    if (rmax <= 1) { TALP_SHAPE_SWITCH(shape, 1, TALP_OCC) }
    else if (rmax <= 2) { TALP_SHAPE_SWITCH(shape, 2, TALP_OCC) }
    else if (rmax <= 4) { TALP_SHAPE_SWITCH(shape, 4, TALP_OCC) }
    else { TALP_SHAPE_SWITCH(shape, 8, TALP_OCC) }
    return 0;
}

int sweep_tile(int shape) {
    if (shape < 0 || shape >= kNumSweepShapes) return 0;
    return 32 * kSweepShapes[shape].items;
}

}  // namespace talp
