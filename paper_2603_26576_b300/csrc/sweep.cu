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
// (blocked, ITEMS odd so the 16-byte shared loads are conflict free), scans
// them serially, and the warp combines lane aggregates with one shuffle
// max-scan per tile.
//
// Arithmetic: a tile is rebased on its first start s0.  When every start and
// end of the tile, and the carries entering it, lie within 2^32 ns of s0
// (any tile whose span is below 4.29 s), the whole tile runs in 32-bit
// unsigned offsets, where max, min and subtraction are single instructions
// and offset 0 stands for "no earlier record".  Otherwise the warp takes the
// exact int64 path.  Both give identical integers.
//
// Regions: the three chain sums of a tile are reduced over the warp once;
// lanes 0 .. 3R-1 each own the accumulator of one (region, chain) and add
// the tile total when the tile's span [s0, max end] lies inside their
// region's window.  Tiles straddling a window boundary recompute their
// pieces clipped to that window.
//
// A warp whose slice starts inside a device segment does not know the
// running max end of the records before its slice; it starts its chains
// empty and the fix-up kernel later subtracts the over-count (the part of the
// slice's new pieces below the true carry), which only touches the records
// whose start lies below the carry.  No warp ever waits on another.
#include "kernels.h"
#include "sweep_core.cuh"

namespace talp {

const SweepShape kSweepShapes[kNumSweepShapes] = {
    {9, 8, 2},   // 288-record tiles, 8 warps, 2 stages, 2 CTAs/SM
    {7, 8, 3},   // 224-record tiles, 8 warps, 3 stages, 2 CTAs/SM
    {11, 8, 2},  // 352-record tiles, 8 warps, 2 stages, 2 CTAs/SM
    {13, 8, 2},  // 416-record tiles, 8 warps, 2 stages, 2 CTAs/SM
};

template <int ITEMS, int WARPS, int STAGES>
struct SweepCfg {
    static constexpr int TILE = 32 * ITEMS;
    static constexpr int SE_BYTES = TILE * 16;
    static constexpr int TAG_BYTES = TILE + 32;                 // 16-byte aligned superset of a tile's tags
    static constexpr int STAGE_BYTES = SE_BYTES + TAG_BYTES;    // multiple of 16
    static constexpr int RAW = STAGES * STAGE_BYTES + STAGES * 8;
    static constexpr int WARP_BYTES = (RAW + 127) / 128 * 128;
    static constexpr int SMEM = WARPS * WARP_BYTES;
};

// The ingest's segments occupy one virtual index space: segment s owns
// [seg_start[s], seg_start[s+1]); its records sit at [seg_start[s],
// seg_rend[s]) and the positions after them are phantoms that only carry the
// segment's fixed cost (descriptor, windows, carries, flush), so that equal
// slices balance records and segment switches alike.
//
// Position of a warp inside its slice: current tile start, current segment,
// end of the current portion (the segment's last record or the slice end).
struct Walk {
    uint64_t pos, seg_end, seg_base;
    uint32_t seg;
};

// Move to the first record at or after w.pos (skipping phantoms and empty
// segments); false when the slice [.., r1) holds no further record.
__device__ __forceinline__ bool walk_enter(Walk& w, const uint64_t* __restrict__ seg_start,
                                           const uint64_t* __restrict__ seg_rend, uint32_t n_segs, uint64_t r1) {
    while (w.seg < n_segs) {
        const uint64_t vs = seg_start[w.seg];
        if (w.pos < vs) w.pos = vs;
        if (w.pos >= r1) return false;
        const uint64_t ve = seg_rend[w.seg];
        if (w.pos < ve) {
            w.seg_base = vs;
            w.seg_end = ve < r1 ? ve : r1;
            return true;
        }
        ++w.seg;
    }
    return false;
}

// Advance past a tile of len records; false when the slice is done.
__device__ __forceinline__ bool walk_advance(Walk& w, uint32_t len, const uint64_t* __restrict__ seg_start,
                                             const uint64_t* __restrict__ seg_rend, uint32_t n_segs, uint64_t r1) {
    w.pos += len;
    if (w.pos < w.seg_end) return true;
    if (w.pos >= r1) return false;
    ++w.seg;
    return walk_enter(w, seg_start, seg_rend, n_segs, r1);
}

// SKIP: the ingest sorts the device segments found out of order and sweeps
// them again from their saved sums, so a warp that finds such a segment out
// of order lets the rest of its part of it stream past uncomputed.  Ingests
// that assert start order launch the instantiation without it.
// Run log of a tile with a descent (first sweep only): j0 = the segment
// position of the lane's first record; last_s = the start before the tile.
// From the lane's 32-bit offsets (the tile's fast path, its buffer already
// handed back to the copy engine) ...
template <int ITEMS>
__device__ __forceinline__ void note_tile_regs(const RunLog& rl, uint32_t seg, uint64_t j0,
                                               const uint32_t (&sr)[ITEMS], int cnt, int64_t s0, int64_t last_s) {
    const int lane = threadIdx.x & 31;
    const uint32_t before = __shfl_up_sync(0xFFFFFFFFu, sr[ITEMS - 1], 1);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        bool desc = false;
        if (i < cnt) desc = i > 0 ? sr[i] < sr[i - 1] : (lane > 0 ? sr[0] < before : s0 < last_s);
        runlog_note(rl, seg, desc && j0 + i > 0, j0 + i);
    }
}

// ... or from the tile in shared memory
template <int ITEMS>
__device__ __forceinline__ void note_tile_smem(const RunLog& rl, uint32_t seg, uint64_t j0, const longlong2* sse,
                                               int base, int cnt, int64_t last_s) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        bool desc = false;
        if (i < cnt) desc = sse[base + i].x < ((i > 0 || lane > 0) ? sse[base + i - 1].x : last_s);
        runlog_note(rl, seg, desc && j0 + i > 0, j0 + i);
    }
}

template <int ITEMS, int WARPS, int STAGES, int RMAX, int MINB, bool SKIP>
__global__ void __launch_bounds__(WARPS * 32, MINB)
    sweep_kernel(const SegDesc* __restrict__ segs, const uint64_t* __restrict__ seg_start,
                 const uint64_t* __restrict__ seg_rend, uint32_t n_segs,
                 WarpRec* __restrict__ wrec, uint32_t* __restrict__ seg_flags, uint32_t* __restrict__ gstatus,
                 int64_t wait_limit, RunLog rl, uint32_t n_chunks, uint32_t* __restrict__ ticket) {
    using C = SweepCfg<ITEMS, WARPS, STAGES>;
    constexpr int TILE = C::TILE;
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    uint8_t* wsm = smem + wid * C::WARP_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wsm + STAGES * C::STAGE_BYTES);

    const uint64_t GW = static_cast<uint64_t>(gridDim.x) * WARPS;
    const uint64_t gw = static_cast<uint64_t>(blockIdx.x) * WARPS + wid;
    const uint64_t N = seg_start[n_segs];
    // Slices of the virtual array: with a ticket, n_chunks equal slices
    // handed to the warps as they come free (so that warps whose slices run
    // slow, e.g. many short segments cut by window boundaries, take fewer);
    // without, one slice per warp.  wrec has one record per slice.
    const uint64_t NCH = ticket ? n_chunks : GW;
    auto next_slice = [&]() -> uint64_t {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(ticket, 1u);
        return __shfl_sync(0xFFFFFFFFu, t, 0);
    };
    auto empty_rec = [&](uint64_t c) {
        if (lane == 0) {
            WarpRec rec;
            rec.head_pos = (N * c) / NCH;
            rec.head_end = rec.head_pos;
            rec.head_seg = NONE;
            rec.tail_seg = NONE;
            rec.head_K = rec.head_M = rec.tail_K = rec.tail_M = NEG_INF;
            wrec[c] = rec;
        }
    };

    if (lane == 0) {
#pragma unroll
        for (int st = 0; st < STAGES; ++st) mbar_init(&bars[st], 1);
        fence_mbar_init();
    }
    __syncwarp();

    // copies issued and tiles consumed over all of the warp's slices (the
    // ring's stage and phase follow from them)
    uint32_t n_issued = 0, n_consumed = 0;
    bool timed_out = false;
    uint32_t* d_status = nullptr;
    uint64_t chunk = ticket ? next_slice() : gw;
    for (; chunk < NCH; chunk = ticket ? next_slice() : NCH) {
    const uint64_t r0 = (N * chunk) / NCH;
    const uint64_t r1 = (N * (chunk + 1)) / NCH;

    // segment containing r0: the last index whose start is <= r0
    uint32_t lo = 0, hi = n_segs;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (seg_start[mid] <= r0) lo = mid; else hi = mid;
    }
    Walk cw;
    cw.pos = r0;
    cw.seg = lo;
    if (r0 >= r1 || !walk_enter(cw, seg_start, seg_rend, n_segs, r1)) {
        empty_rec(chunk);   // the slice holds no record (empty or phantom positions only)
        continue;
    }

    // ---- producer (lane 0): its own walk over the same tile sequence
    Walk iw = cw;
    bool iw_done = false;
    uint32_t iw_cached = NONE;
    const int64_t* iw_se = nullptr;
    const uint8_t* iw_tag = nullptr;
    uintptr_t iw_lim = 0;

    auto issue = [&](int st) {
        if (iw_cached != iw.seg) {
            const SegDesc& d = segs[iw.seg];
            iw_se = d.se;
            iw_tag = d.tag;
            iw_lim = reinterpret_cast<uintptr_t>(d.tag_limit);
            iw_cached = iw.seg;
        }
        const uint64_t off = iw.pos - iw.seg_base;
        const uint64_t rem = iw.seg_end - iw.pos;
        const uint32_t len = rem < static_cast<uint64_t>(TILE) ? static_cast<uint32_t>(rem) : TILE;
        uint8_t* stage = wsm + st * C::STAGE_BYTES;
        const uintptr_t A = reinterpret_cast<uintptr_t>(iw_tag + off);
        const uintptr_t tlo = A & ~static_cast<uintptr_t>(15);
        uintptr_t thi = (A + len + 15) & ~static_cast<uintptr_t>(15);
        if (thi > iw_lim) thi = iw_lim;
        const uint32_t tag_bytes = thi > tlo ? static_cast<uint32_t>(thi - tlo) : 0u;
        mbar_arrive_expect_tx(&bars[st], len * 16u + tag_bytes);
        tma_load_1d(stage, iw_se + 2 * off, len * 16u, &bars[st]);
        if (tag_bytes) tma_load_1d(stage + C::SE_BYTES, reinterpret_cast<const void*>(tlo), tag_bytes, &bars[st]);
        ++n_issued;
        if (!walk_advance(iw, len, seg_start, seg_rend, n_segs, r1)) iw_done = true;
    };

    if (lane == 0) {
        for (int st = 0; st < STAGES && !iw_done; ++st) issue(static_cast<int>(n_issued % STAGES));
    }

    // ---- consumers (all lanes): the same walk
    if (lane == 0) {
        wrec[chunk].head_pos = cw.pos;
        wrec[chunk].head_seg = cw.seg;
        wrec[chunk].head_end = cw.seg_end;
    }
    bool first_portion = true;

    // per portion
    const uint8_t* d_tag = nullptr;
    uintptr_t d_lim = 0;
    int64_t* d_sums = nullptr;
    int64_t* d_cout = nullptr;
    int d_R = 0;
    bool d_host = false;
    int64_t wa = 0, wb = 0;   // lane j < 3R: window of region j / 3
    int64_t acc = 0;          // lane j < 3R: sum of chain j % 3 in region j / 3
    int64_t carryK = NEG_INF, carryM = NEG_INF, last_s = NEG_INF;
    uint32_t pbad = 0;
    bool d_sortable = false;  // SKIP: the segment may be sorted and swept again
    bool skip_seg = false;    // SKIP, warp-uniform: this warp found it out of order
    bool portion_open = false;
    const int lchain = lane % 3;

    auto release = [&](int st) {
        __syncwarp();
        if (lane == 0) {
            fence_proxy_async_smem();
            if (!iw_done) issue(st);
        }
    };

    while (true) {
        if (!portion_open) {
            const SegDesc& d = segs[cw.seg];
            d_tag = d.tag;
            d_lim = reinterpret_cast<uintptr_t>(d.tag_limit);
            d_sums = d.sums;
            d_status = d.status;
            d_cout = d.carry_out;
            d_R = d.R;
            d_host = d.is_host != 0;
            if (lane < 3 * d_R) {
                wa = d.win[2 * (lane / 3)];
                wb = d.win[2 * (lane / 3) + 1];
            }
            acc = 0;
            pbad = 0;
            if constexpr (SKIP) {
                d_sortable = !d_host && (d.pad[0] & kSegSortable) != 0;
                skip_seg = false;
            }
            if (!d_host && cw.pos == cw.seg_base) {
                carryK = d.carry_in[0];
                carryM = d.carry_in[1];
                last_s = d.carry_in[2];
            } else {
                carryK = carryM = last_s = NEG_INF;
            }
            portion_open = true;
        }
        const int st = static_cast<int>(n_consumed % STAGES);
        const uint32_t ph = (n_consumed / STAGES) & 1u;
        const bool ok = mbar_wait_bounded(&bars[st], ph, wait_limit);
        if (__any_sync(0xFFFFFFFFu, !ok)) {
            timed_out = true;
            break;
        }
        uint8_t* stage = wsm + st * C::STAGE_BYTES;
        const longlong2* sse = reinterpret_cast<const longlong2*>(stage);
        const uint64_t off = cw.pos - cw.seg_base;
        const uint64_t rem = cw.seg_end - cw.pos;
        const int len = rem < static_cast<uint64_t>(TILE) ? static_cast<int>(rem) : TILE;
        if constexpr (SKIP) {
            if (skip_seg) {   // the rest of a segment that will be sorted and swept again
                if (rl.n) {
                    // only scanned for the run log, unless the segment has
                    // too many runs for it already
                    uint32_t many = 0;
                    if (lane == 0) many = *static_cast<volatile uint32_t*>(&rl.n[cw.seg]) >= kMaxRuns;
                    if (!__shfl_sync(0xFFFFFFFFu, many, 0)) {
                        const int b0 = lane * ITEMS;
                        note_tile_smem<ITEMS>(rl, cw.seg, off + b0, sse, b0, max(0, min(ITEMS, len - b0)), last_s);
                    }
                    last_s = sse[len - 1].x;
                }
                release(st);
                ++n_consumed;
                const bool seg_done = cw.pos + static_cast<uint64_t>(len) == cw.seg_end;
                const uint32_t seg_now = cw.seg;
                const bool more = walk_advance(cw, static_cast<uint32_t>(len), seg_start, seg_rend, n_segs, r1);
                if (seg_done) {   // its flags go out; its sums and carries are restored before the re-sweep
                    const uint32_t bits = __reduce_or_sync(0xFFFFFFFFu, pbad);
                    if (lane == 0) {
                        if (bits) {
                            atomicOr(d_status, bits);
                            atomicOr(&seg_flags[seg_now], bits);
                        }
                        if (!more) wrec[chunk].tail_seg = seg_now;
                    }
                    first_portion = false;
                    portion_open = false;
                }
                if (!more) break;
                continue;
            }
        }
        const uintptr_t A = reinterpret_cast<uintptr_t>(d_tag + off);
        uint8_t* stag = stage + C::SE_BYTES + static_cast<int>(A & 15u);
        const int direct_from =
            d_lim > A ? static_cast<int>(min(static_cast<uint64_t>(d_lim - A), static_cast<uint64_t>(len))) : 0;
        if (direct_from < len) {
            // the last bytes of the tag array lie past the last 16-byte
            // boundary the bulk copy may touch: fetch them directly
            for (int k = direct_from + lane; k < len; k += 32) stag[k] = d_tag[off + k];
            __syncwarp();
        }

        const int base = lane * ITEMS;
        const int cnt = max(0, min(ITEMS, len - base));
        const int64_t s0 = sse[0].x;
        const int64_t tile_last_s = sse[len - 1].x;
        uint32_t sr[ITEMS], er[ITEMS], tg[ITEMS];
        uint32_t hib = 0;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if (i < cnt) {
                const longlong2 v = sse[base + i];
                const int64_t ds = v.x - s0, de = v.y - s0;
                sr[i] = static_cast<uint32_t>(ds);
                er[i] = static_cast<uint32_t>(de);
                hib |= static_cast<uint32_t>(ds >> 32) | static_cast<uint32_t>(de >> 32);
                tg[i] = stag[base + i];
            } else {
                sr[i] = er[i] = tg[i] = 0;
            }
        }
        uint32_t bad = 0;
        if (!d_host && cnt > 0) {
            const int64_t prev = lane == 0 ? last_s : sse[base - 1].x;
            bad |= (sse[base].x < prev) ? ST_UNSORTED : 0u;
        }
        const bool carry_ok = (carryK <= s0 || ((carryK - s0) >> 32) == 0) &&
                              (carryM <= s0 || ((carryM - s0) >> 32) == 0);
        const bool fast = __all_sync(0xFFFFFFFFu, hib == 0) && carry_ok;
        if (fast) release(st);

        // tile totals of the three sums (warp-uniform) and the tile span
        int64_t tot0 = 0, tot1 = 0, tot2 = 0;
        int64_t span_lo = s0, span_hi = s0;
        if (fast) {
            uint32_t s1 = 0, s2 = 0, s3 = 0;   // device: K, M, all chain sums of the lane
            uint32_t lo32 = 0, hi32 = 0;
            uint64_t h0 = 0, h1 = 0, h2 = 0;   // host: U, W, MPI sums of the lane
            uint32_t xK = 0, xM = 0;
            const bool full = len == TILE;     // warp-uniform: no per-record guards
            if (!d_host) {
                const uint32_t cK = carryK <= s0 ? 0u : static_cast<uint32_t>(carryK - s0);
                const uint32_t cM = carryM <= s0 ? 0u : static_cast<uint32_t>(carryM - s0);
                uint32_t aK = 0, aM = 0;
                bool okE = true, okS = true, okK = true;
                if (full) dev_pass1<ITEMS, true>(sr, er, tg, cnt, aK, aM, okE, okS, okK);
                else dev_pass1<ITEMS, false>(sr, er, tg, cnt, aK, aM, okE, okS, okK);
                bad |= (okE ? 0u : ST_BAD_END) | (okK ? 0u : ST_BAD_KIND) | (okS ? 0u : ST_UNSORTED);
                if constexpr (SKIP) {
                    if (rl.n && d_sortable && __any_sync(0xFFFFFFFFu, (bad & ST_UNSORTED) != 0u))
                        note_tile_regs<ITEMS>(rl, cw.seg, off + base, sr, cnt, s0, last_s);
                }
                uint32_t iK = aK, iM = aM;
#pragma unroll
                for (int dd = 1; dd < 32; dd <<= 1) {
                    const uint32_t tk = __shfl_up_sync(0xFFFFFFFFu, iK, dd);
                    const uint32_t tm = __shfl_up_sync(0xFFFFFFFFu, iM, dd);
                    if (lane >= dd) {
                        iK = umax(iK, tk);
                        iM = umax(iM, tm);
                    }
                }
                xK = __shfl_up_sync(0xFFFFFFFFu, iK, 1);
                xM = __shfl_up_sync(0xFFFFFFFFu, iM, 1);
                if (lane == 0) xK = xM = 0u;
                xK = umax(xK, cK);
                xM = umax(xM, cM);
                const uint32_t tK = __shfl_sync(0xFFFFFFFFu, iK, 31);
                const uint32_t tM = __shfl_sync(0xFFFFFFFFu, iM, 31);
                if (tK) carryK = max64(carryK, s0 + tK);
                if (tM) carryM = max64(carryM, s0 + tM);
                hi32 = umax(tK, tM);
                if (full) pieces32<ITEMS, true>(sr, er, tg, cnt, xK, xM, 0u, 0xFFFFFFFFu, s1, s2, s3);
                else pieces32<ITEMS, false>(sr, er, tg, cnt, xK, xM, 0u, 0xFFFFFFFFu, s1, s2, s3);
                tot0 = __reduce_add_sync(0xFFFFFFFFu, s1);
                tot1 = __reduce_add_sync(0xFFFFFFFFu, s2);
                tot2 = __reduce_add_sync(0xFFFFFFFFu, s3);
            } else {
                lo32 = 0xFFFFFFFFu;
                bool okE = true, okK = true;
                if (full) host_pass<ITEMS, true>(sr, er, tg, cnt, 0u, 0xFFFFFFFFu, h0, h1, h2, lo32, hi32, okE, okK);
                else host_pass<ITEMS, false>(sr, er, tg, cnt, 0u, 0xFFFFFFFFu, h0, h1, h2, lo32, hi32, okE, okK);
                bad |= (okE ? 0u : ST_BAD_END) | (okK ? 0u : ST_BAD_KIND);
                tot0 = warp_sum_u64_small(h0);
                tot1 = warp_sum_u64_small(h1);
                tot2 = warp_sum_u64_small(h2);
                lo32 = __reduce_min_sync(0xFFFFFFFFu, lo32);
                hi32 = __reduce_max_sync(0xFFFFFFFFu, hi32);
                span_lo = s0 + lo32;
            }
            span_hi = s0 + hi32;
            // classification of the tile span against the lane's region
            const bool mine = lane < 3 * d_R;
            const bool inside = mine && wa <= span_lo && span_hi <= wb;
            const bool outside = mine && (span_hi <= wa || span_lo >= wb);
            if (inside) acc += lchain == 0 ? tot0 : (lchain == 1 ? tot1 : tot2);
            uint32_t sb = __ballot_sync(0xFFFFFFFFu, mine && lchain == 0 && !inside && !outside);
            // windows cutting the tile: the pieces' starts do not depend on
            // the window, so the shapes with registers to spare (the ones
            // short segments use) work them out once (over sr, no longer
            // needed as starts) and each window only clips
            constexpr bool kStarts = ITEMS <= 9;
            uint32_t pO[ITEMS];
            if (kStarts && sb && !d_host) piece_starts<ITEMS>(sr, pO, er, tg, cnt, xK, xM);
            while (sb) {
                const int src = __ffs(sb) - 1;
                sb &= sb - 1;
                const int64_t a64 = shfl64(wa, src), b64 = shfl64(wb, src);
                const uint32_t a = rel_sat(a64, s0), b = rel_sat(b64, s0);
                int64_t c0, c1, c2;
                if (!d_host) {
                    uint32_t k1 = 0, k2 = 0, k3 = 0;
                    if (kStarts) clip_pieces<ITEMS>(sr, pO, er, tg, cnt, a, b, k1, k2, k3);
                    else pieces32<ITEMS, false>(sr, er, tg, cnt, xK, xM, a, b, k1, k2, k3);
                    c0 = __reduce_add_sync(0xFFFFFFFFu, k1);
                    c1 = __reduce_add_sync(0xFFFFFFFFu, k2);
                    c2 = __reduce_add_sync(0xFFFFFFFFu, k3);
                } else {
                    uint64_t g0 = 0, g1 = 0, g2 = 0;
                    uint32_t l2 = 0, h2x = 0;
                    bool e2 = true, k2x = true;
                    host_pass<ITEMS, false>(sr, er, tg, cnt, a, b, g0, g1, g2, l2, h2x, e2, k2x);
                    c0 = warp_sum_u64_small(g0);
                    c1 = warp_sum_u64_small(g1);
                    c2 = warp_sum_u64_small(g2);
                }
                if (lane / 3 == src / 3 && mine) acc += lchain == 0 ? c0 : (lchain == 1 ? c1 : c2);
            }
        } else {
            // exact int64 path (a tile spanning 2^32 ns or more)
            int64_t k0 = 0, k1 = 0, k2 = 0;
            int64_t xK = NEG_INF, xM = NEG_INF;
            int64_t lo64 = INT64_MAX, hi64 = NEG_INF;
            if (!d_host) {
                int64_t aK = NEG_INF, aM = NEG_INF;
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    if (i < cnt) {
                        const longlong2 v = sse[base + i];
                        const uint32_t kind = tg[i] >> 5;
                        bad |= (v.y < v.x) ? ST_BAD_END : 0u;
                        bad |= (kind > 4u) ? ST_BAD_KIND : 0u;
                        if (i > 0) bad |= (v.x < sse[base + i - 1].x) ? ST_UNSORTED : 0u;
                        if (kind == 0u) aK = max64(aK, v.y); else aM = max64(aM, v.y);
                    }
                }
                int64_t iK = aK, iM = aM;
                warp_incl_max2(iK, iM, lane);
                xK = shfl_up64(iK, 1);
                xM = shfl_up64(iM, 1);
                if (lane == 0) xK = xM = NEG_INF;
                xK = max64(xK, carryK);
                xM = max64(xM, carryM);
                const int64_t tK = shfl64(iK, 31), tM = shfl64(iM, 31);
                carryK = max64(carryK, tK);
                carryM = max64(carryM, tM);
                lo64 = s0;
                hi64 = max64(tK, tM);
                pieces64<ITEMS>(sse, base, tg, cnt, xK, xM, NEG_INF, INT64_MAX, k0, k1, k2);
            } else {
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    if (i < cnt) {
                        const longlong2 v = sse[base + i];
                        const uint32_t q = tg[i];
                        bad |= (v.y < v.x) ? ST_BAD_END : 0u;
                        bad |= (q > 2u) ? ST_BAD_KIND : 0u;
                        const int64_t l = max64(v.y - v.x, 0);
                        k0 += q == 0u ? l : 0;
                        k1 += q == 1u ? l : 0;
                        k2 += q == 2u ? l : 0;
                        lo64 = min64(lo64, v.x);
                        hi64 = max64(hi64, v.y);
                    }
                }
#pragma unroll
                for (int m = 16; m > 0; m >>= 1) {
                    lo64 = min64(lo64, shfl_xor64(lo64, m));
                    hi64 = max64(hi64, shfl_xor64(hi64, m));
                }
            }
            tot0 = warp_sum64(k0);
            tot1 = warp_sum64(k1);
            tot2 = warp_sum64(k2);
            span_lo = lo64;
            span_hi = hi64;
            const bool mine = lane < 3 * d_R;
            const bool inside = mine && wa <= span_lo && span_hi <= wb;
            const bool outside = mine && (span_hi <= wa || span_lo >= wb);
            if (inside) acc += lchain == 0 ? tot0 : (lchain == 1 ? tot1 : tot2);
            uint32_t sb = __ballot_sync(0xFFFFFFFFu, mine && lchain == 0 && !inside && !outside);
            while (sb) {
                const int src = __ffs(sb) - 1;
                sb &= sb - 1;
                const int64_t a = shfl64(wa, src), b = shfl64(wb, src);
                int64_t c0 = 0, c1 = 0, c2 = 0;
                if (!d_host) {
                    pieces64<ITEMS>(sse, base, tg, cnt, xK, xM, a, b, c0, c1, c2);
                } else {
#pragma unroll
                    for (int i = 0; i < ITEMS; ++i) {
                        if (i < cnt) {
                            const longlong2 v = sse[base + i];
                            const uint32_t q = tg[i];
                            const int64_t l = max64(min64(v.y, b) - max64(v.x, a), 0);
                            c0 += q == 0u ? l : 0;
                            c1 += q == 1u ? l : 0;
                            c2 += q == 2u ? l : 0;
                        }
                    }
                }
                c0 = warp_sum64(c0);
                c1 = warp_sum64(c1);
                c2 = warp_sum64(c2);
                if (lane / 3 == src / 3 && mine) acc += lchain == 0 ? c0 : (lchain == 1 ? c1 : c2);
            }
            if constexpr (SKIP) {
                if (rl.n && d_sortable && !d_host && __any_sync(0xFFFFFFFFu, (bad & ST_UNSORTED) != 0u))
                    note_tile_smem<ITEMS>(rl, cw.seg, off + base, sse, base, cnt, last_s);
            }
            release(st);
        }
        if constexpr (SKIP) {
            if (d_sortable && __any_sync(0xFFFFFFFFu, (bad & ST_UNSORTED) != 0u)) skip_seg = true;
        }
        ++n_consumed;
        pbad |= bad;
        last_s = tile_last_s;

        // close the portion when the segment's records (or the slice) end
        const bool seg_done = cw.pos + static_cast<uint64_t>(len) == cw.seg_end;
        const uint32_t seg_now = cw.seg;
        const bool more = walk_advance(cw, static_cast<uint32_t>(len), seg_start, seg_rend, n_segs, r1);
        const bool slice_done = !more;
        if (seg_done) {
            if (lane < 3 * d_R && acc != 0) atomic_add64(&d_sums[lane], acc);
            const uint32_t bits = __reduce_or_sync(0xFFFFFFFFu, pbad);
            if (lane == 0) {
                if (bits) {
                    atomicOr(d_status, bits);
                    atomicOr(&seg_flags[seg_now], bits);
                }
                if (!d_host) {
                    atomic_max64(&d_cout[0], carryK);
                    atomic_max64(&d_cout[1], carryM);
                    atomic_max64(&d_cout[2], last_s);
                }
                if (first_portion) {
                    wrec[chunk].head_K = carryK;
                    wrec[chunk].head_M = carryM;
                }
                if (slice_done) {
                    wrec[chunk].tail_seg = seg_now;
                    wrec[chunk].tail_K = carryK;
                    wrec[chunk].tail_M = carryM;
                }
            }
            first_portion = false;
            portion_open = false;
        }
        if (slice_done) break;
    }
    if (timed_out) break;
    }   // slices

    if (timed_out) {
        if (lane == 0) {
            atomicOr(gstatus, ST_TIMEOUT);
            if (d_status) atomicOr(d_status, ST_TIMEOUT);
            // let the copies still in flight land before the CTA's shared memory goes away
            for (uint32_t t = n_consumed; t < n_issued; ++t)
                (void)mbar_wait_bounded(&bars[t % STAGES], (t / STAGES) & 1u, kDrainWaitCycles);
            wrec[chunk].head_seg = NONE;
            wrec[chunk].tail_seg = NONE;
        }
        // every slice's record is written, swept or not (the fix-up reads them all)
        if (ticket)
            for (chunk = next_slice(); chunk < NCH; chunk = next_slice()) empty_rec(chunk);
    }
}

// ---------------------------------------------------------------- dispatch

// The dynamic shared-memory opt-in of one instantiation, set once per
// process (sizing an ingest does it, so no attribute call happens while a
// launch sequence is being captured into a graph).
template <int ITEMS, int WARPS, int STAGES, int RMAX>
static cudaError_t ensure_smem_attr() {
    using C = SweepCfg<ITEMS, WARPS, STAGES>;
    constexpr int MINB = WARPS == 8 ? 2 : 3;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(sweep_kernel<ITEMS, WARPS, STAGES, RMAX, MINB, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(sweep_kernel<ITEMS, WARPS, STAGES, RMAX, MINB, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    return cudaSuccess;
}

template <int ITEMS, int WARPS, int STAGES, int RMAX>
static cudaError_t launch_t(int grid, const SegDesc* segs, const uint64_t* seg_start, const uint64_t* seg_rend,
                            uint32_t n_segs,
                            WarpRec* wrec, uint32_t* seg_flags, uint32_t* gstatus, int64_t wait_limit,
                            bool skip_sorted_out, RunLog rl, uint32_t n_slices, uint32_t* ticket,
                            cudaStream_t stream) {
    using C = SweepCfg<ITEMS, WARPS, STAGES>;
    constexpr int MINB = WARPS == 8 ? 2 : 3;
    auto k = skip_sorted_out ? sweep_kernel<ITEMS, WARPS, STAGES, RMAX, MINB, true>
                             : sweep_kernel<ITEMS, WARPS, STAGES, RMAX, MINB, false>;
    cudaError_t e = ensure_smem_attr<ITEMS, WARPS, STAGES, RMAX>();
    if (e != cudaSuccess) return e;
    k<<<grid, WARPS * 32, C::SMEM, stream>>>(segs, seg_start, seg_rend, n_segs, wrec, seg_flags, gstatus,
                                              wait_limit, rl, n_slices, ticket);
    return cudaGetLastError();
}

template <int ITEMS, int WARPS, int STAGES, int RMAX>
static int occupancy_t() {
    using C = SweepCfg<ITEMS, WARPS, STAGES>;
    constexpr int MINB = WARPS == 8 ? 2 : 3;
    auto k = sweep_kernel<ITEMS, WARPS, STAGES, RMAX, MINB, false>;
    if (ensure_smem_attr<ITEMS, WARPS, STAGES, RMAX>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, WARPS * 32, C::SMEM) != cudaSuccess) return 0;
    return n;
}

#define TALP_SHAPE_SWITCH(shape, RM, CALL)                \
    switch (shape) {                                      \
        case 0: return CALL(9, 8, 2, RM);                 \
        case 1: return CALL(7, 8, 3, RM);                 \
        case 2: return CALL(11, 8, 2, RM);                \
        case 3: return CALL(13, 8, 2, RM);                \
        default: break;                                   \
    }

#define TALP_LAUNCH(I, W, S, RM) \
    launch_t<I, W, S, RM>(grid, segs, seg_start, seg_rend, n_segs, wrec, seg_flags, gstatus, wait_limit, \
                          skip_sorted_out, rl, n_slices, ticket, stream)
#define TALP_OCC(I, W, S, RM) occupancy_t<I, W, S, RM>()

// The region count no longer shapes the kernel's registers (each lane owns
// one (region, chain) accumulator), so one instantiation per shape serves
// every R <= 8.
cudaError_t launch_sweep(int shape, int rmax, int grid, const SegDesc* segs, const uint64_t* seg_start,
                         const uint64_t* seg_rend, uint32_t n_segs, WarpRec* wrec, uint32_t* seg_flags,
                         uint32_t* gstatus, int64_t wait_limit, bool skip_sorted_out, RunLog rl,
                         uint32_t n_slices, uint32_t* ticket, cudaStream_t stream) {
    (void)rmax;
    TALP_SHAPE_SWITCH(shape, 8, TALP_LAUNCH)
    return cudaErrorInvalidValue;
}

int sweep_ctas_per_sm(int shape, int rmax) {
    (void)rmax;
    TALP_SHAPE_SWITCH(shape, 8, TALP_OCC)
    return 0;
}

int sweep_tile(int shape) {
    if (shape < 0 || shape >= kNumSweepShapes) return 0;
    return 32 * kSweepShapes[shape].items;
}

}  // namespace talp
