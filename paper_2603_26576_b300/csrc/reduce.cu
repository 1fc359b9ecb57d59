// Fix-up of slice boundaries, state preparation, and the final reduction
// into the Eq. 1 / Eqs. 6-12 metrics.
#include "kernels.h"

namespace talp {

// ------------------------------------------------------------------ fix-up
//
// A sweep warp whose slice starts inside a device segment ran its three
// chains from an empty carry.  Its new pieces are then too long exactly by
// their part below the true carry C (the largest end before the slice), so
// the fix-up subtracts |piece ∩ (-inf, C) ∩ [a, b)| for each chain and region.
// Only records starting below C have such a part; with the records in start
// order they form a prefix of the slice, usually a handful of records.
// C comes from the running state of earlier ingests and from the portions of
// the same segment owned by the preceding warps (a warp-parallel walk back).
// One warp per sweep warp; nothing waits on anything.
__global__ void __launch_bounds__(256) fixup_kernel(const SegDesc* __restrict__ segs,
                                                    const uint64_t* __restrict__ seg_start,
                                                    const WarpRec* __restrict__ wrec, uint32_t n_wrec,
                                                    uint32_t* __restrict__ seg_flags, bool skip_resorted,
                                                    RunLog rl) {
    constexpr int RM = 8;
    const int lane = threadIdx.x & 31;
    const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= n_wrec) return;
    const WarpRec rec = wrec[w];
    if (rec.head_seg == NONE) return;
    const uint32_t seg = rec.head_seg;
    const SegDesc d = segs[seg];
    if (d.is_host) return;
    const uint64_t sbase = seg_start[seg];
    if (rec.head_pos <= sbase) return;

    const uint64_t off0 = rec.head_pos - sbase;
    if (lane == 0 && d.se[2 * off0] < d.se[2 * (off0 - 1)]) {
        atomicOr(d.status, ST_UNSORTED);
        atomicOr(&seg_flags[seg], ST_UNSORTED);
        // the one pair of records the sweep did not compare: into the run log
        if (rl.n && (d.pad[0] & kSegSortable)) {
            const uint32_t slot = atomicAdd(&rl.n[seg], 1u);
            if (slot < static_cast<uint32_t>(kMaxRuns - 1)) rl.pos[static_cast<uint64_t>(seg) * kMaxRuns + slot] = off0;
        }
    }
    // a segment already found out of order and allowed to sort is sorted and
    // swept again from its saved sums: correcting this pass is wasted work
    // (and, its records not being in order, not a short prefix)
    if (skip_resorted && (d.pad[0] & kSegSortable) && (seg_flags[seg] & ST_UNSORTED)) return;

    // carry: running state + tails of the preceding warps inside this segment
    int64_t CK = d.carry_in[0];
    int64_t CM = d.carry_in[1];
    for (int64_t b = static_cast<int64_t>(w) - 1; b >= 0; b -= 32) {
        const int64_t idx = b - lane;
        bool stop = true;
        int64_t tk = NEG_INF, tm = NEG_INF;
        if (idx >= 0) {
            const WarpRec p = wrec[idx];
            if (p.tail_seg == seg) {
                tk = p.tail_K;
                tm = p.tail_M;
            }
            stop = (p.head_seg != NONE) && !(p.head_seg == seg && p.head_pos > sbase);
        }
        const uint32_t sm = __ballot_sync(0xFFFFFFFFu, stop);
        const int first = sm ? (__ffs(sm) - 1) : 31;
        if (lane > first) {
            tk = NEG_INF;
            tm = NEG_INF;
        }
        CK = max64(CK, warp_max64(tk));
        CM = max64(CM, warp_max64(tm));
        if (sm) break;
    }
    const int64_t CA = max64(CK, CM);
    if (CA == NEG_INF) return;

    int64_t sub[RM][3];
#pragma unroll
    for (int r = 0; r < RM; ++r) sub[r][0] = sub[r][1] = sub[r][2] = 0;
    int64_t Kl = NEG_INF, Ml = NEG_INF;
    for (uint64_t p = rec.head_pos; p < rec.head_end; p += 32) {
        const uint64_t j = p + lane;
        const bool valid = j < rec.head_end;
        int64_t s = 0, e = 0;
        uint32_t kind = 0;
        if (valid) {
            const uint64_t o = j - sbase;
            s = d.se[2 * o];
            e = d.se[2 * o + 1];
            kind = d.tag[o] >> 5;
        }
        const bool isK = kind == 0u;
        int64_t iK = (valid && isK) ? e : NEG_INF;
        int64_t iM = (valid && !isK) ? e : NEG_INF;
        warp_incl_max2(iK, iM, lane);
        int64_t xK = shfl_up64(iK, 1), xM = shfl_up64(iM, 1);
        if (lane == 0) {
            xK = NEG_INF;
            xM = NEG_INF;
        }
        xK = max64(xK, Kl);
        xM = max64(xM, Ml);
        Kl = max64(Kl, shfl64(iK, 31));
        Ml = max64(Ml, shfl64(iM, 31));
        if (valid && s < CA) {
            // a chain's over-count exists only below its own carry; a chain
            // without carry (NEG_INF) has none (and must not enter the
            // subtraction, which would overflow)
            const int64_t CO = isK ? CK : CM;
            const bool own = s < CO;
            const int64_t pA = max64(s, max64(xK, xM));
            const int64_t pO = max64(s, isK ? xK : xM);
            const int64_t eA = min64(e, CA);
            const int64_t eO = own ? min64(e, CO) : s;
#pragma unroll
            for (int r = 0; r < RM; ++r) {
                if (r < d.R) {
                    const int64_t a = d.win[2 * r], b = d.win[2 * r + 1];
                    sub[r][2] += max64(min64(eA, b) - max64(pA, a), 0);
                    if (own) sub[r][isK ? 0 : 1] += max64(min64(eO, b) - max64(pO, a), 0);
                }
            }
        }
        if (__any_sync(0xFFFFFFFFu, valid && s >= CA)) break;
    }
#pragma unroll
    for (int r = 0; r < RM; ++r) {
        if (r < d.R) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t v = warp_sum64(sub[r][c]);
                if (lane == 0 && v != 0) atomic_add64(&d.sums[3 * r + c], -v);
            }
        }
    }
}

cudaError_t launch_fixup(const SegDesc* segs, const uint64_t* seg_start, const WarpRec* wrec, uint32_t n_wrec,
                         uint32_t* seg_flags, bool skip_resorted, RunLog rl, cudaStream_t stream) {
    if (n_wrec == 0) return cudaSuccess;
    const int wpb = 8;
    const int grid = static_cast<int>((n_wrec + wpb - 1) / wpb);
    fixup_kernel<<<grid, wpb * 32, 0, stream>>>(segs, seg_start, wrec, n_wrec, seg_flags, skip_resorted, rl);
    return cudaGetLastError();
}

// -------------------------------------------------------------------- prep
// Zero the sums of freshly ingested traces, reset or copy running state.
__global__ void __launch_bounds__(256) prep_kernel(const FillJob* __restrict__ jobs, uint32_t n_jobs) {
    for (uint32_t j = blockIdx.y; j < n_jobs; j += gridDim.y) {
        const FillJob job = jobs[j];
        for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < job.count; i += 256ull * gridDim.x)
            job.ptr[i] = job.src ? (job.value ? job.ptr[i] + job.src[i] : job.src[i]) : job.value;
    }
}

cudaError_t launch_prep(const FillJob* jobs, uint32_t n_jobs, cudaStream_t stream) {
    if (n_jobs == 0) return cudaSuccess;
    // a few large jobs (one trace) get 8 CTAs each; many small ones (a
    // batch of traces) one, so that the launch is not thousands of CTAs with
    // nothing to do
    dim3 grid(n_jobs >= 1024 ? 1 : 8, n_jobs < 65535 ? n_jobs : 65535);
    prep_kernel<<<grid, 256, 0, stream>>>(jobs, n_jobs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- finalize
//
// One warp per (trace, region): reduce the per-rank host sums and per-device
// unions into E and the sums/maxima, then form the nine ratios in FP64 with
// the fixed order num / (k * den) (forms with n or m) or num / den, round to
// nearest, no contraction: Eqs. 6-8 (host tree) and 9-12 (device tree).
__device__ __forceinline__ double ratio_k(int64_t num, int64_t k, int64_t den) {
    if (k == 0 || den == 0) return 1.0;
    return __ddiv_rn(__ll2double_rn(num), __dmul_rn(__ll2double_rn(k), __ll2double_rn(den)));
}
__device__ __forceinline__ double ratio(int64_t num, int64_t den) {
    if (den == 0) return 1.0;
    return __ddiv_rn(__ll2double_rn(num), __ll2double_rn(den));
}

// The nine ratios from the region's integer aggregates (o.flags holds the
// status bits on entry; EMPTY and NO_DEVICES are set here).  E = 0 gives
// EMPTY with every ratio 1; 0/0 := 1 for the factors.
__device__ __forceinline__ void form_ratios(MetricsOut& o) {
    const int64_t E = o.elapsed_ns, n = o.n_ranks, m = o.m_devices;
    const int64_t sU = o.sum_useful, sW = o.sum_offload, maxUW = o.max_useful_offload;
    const int64_t sK = o.sum_kernel, maxK = o.max_kernel, maxB = o.max_busy;
    if (E == 0) {
        o.flags |= 0x1u;
        if (m == 0) o.flags |= 0x4u;
        o.host_pe = o.host_mpi_pe = o.host_mpi_lb = o.host_mpi_ce = o.host_oe = 1.0;
        o.dev_pe = o.dev_lb = o.dev_ce = o.dev_oe = 1.0;
        return;
    }
    o.host_pe = ratio_k(sU, E, n);          // Eq. 6
    o.host_mpi_pe = ratio_k(sU + sW, E, n); // Eq. 7
    o.host_mpi_lb = ratio_k(sU + sW, n, maxUW);
    o.host_mpi_ce = ratio(maxUW, E);
    o.host_oe = ratio(sU, sU + sW);         // Eq. 8
    if (m == 0) {
        o.flags |= 0x4u;
        o.dev_pe = o.dev_lb = o.dev_ce = o.dev_oe = 1.0;
        return;
    }
    o.dev_pe = ratio_k(sK, E, m);           // Eq. 9
    o.dev_lb = ratio_k(sK, m, maxK);        // Eq. 10
    o.dev_ce = ratio(maxK, maxB);           // Eq. 11
    o.dev_oe = ratio(maxB, E);              // Eq. 12
}

template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v = op(v, static_cast<T>(__shfl_xor_sync(0xFFFFFFFFu, v, m)));
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T r = sh[0];
    for (int i = 1; i < static_cast<int>(blockDim.x >> 5); ++i) r = op(r, sh[i]);
    return r;
}

// One warp per (trace, region) job, 8 jobs per CTA: the unit sums of the
// job are read once and reduced by warp shuffles (integer sums and maxima,
// so the order of the reduction does not matter).
constexpr int kFinWarps = 8;
__global__ void __launch_bounds__(32 * kFinWarps) finalize_kernel(const FinalizeJob* __restrict__ jobs,
                                                                  uint32_t n_jobs) {
    const int lane = threadIdx.x & 31;
    const uint32_t jx = blockIdx.x * kFinWarps + (threadIdx.x >> 5);
    if (jx >= n_jobs) return;
    const FinalizeJob job = jobs[jx];
    const TraceDev t = *job.t;
    const uint32_t r = job.region;
    const uint32_t R = t.R;
    auto mx = [](long long a, long long b) { return a > b ? a : b; };

    long long E = 0, sU = 0, sW = 0, sP = 0, maxUW = 0;
    uint32_t not_tiled = 0;
    for (uint32_t i = lane; i < t.n; i += 32) {
        const int64_t* h = t.hsum + (static_cast<uint64_t>(i) * R + r) * 3;
        const int64_t U = h[0], W = h[1], P = h[2];
        const int64_t* wv = t.hwin + (static_cast<uint64_t>(i) * R + r) * 2;
        E = mx(E, U + W + P);
        sU += U;
        sW += W;
        sP += P;
        maxUW = mx(maxUW, U + W);
        if (U + W + P != wv[1] - wv[0]) not_tiled = 1;
    }
    long long sK = 0, maxK = 0, maxB = 0, sM = 0, sIdle = 0, sHid = 0;
    for (uint32_t g = lane; g < t.m; g += 32) {
        const int64_t* u = t.dsum + (static_cast<uint64_t>(g) * R + r) * 3;
        const int64_t K = u[0], UM = u[1], B = u[2];
        const int64_t DM = B - K;
        const int64_t* wv = t.hwin + (static_cast<uint64_t>(t.dev_rank[g]) * R + r) * 2;
        sK += K;
        maxK = mx(maxK, K);
        maxB = mx(maxB, K + DM);
        sM += DM;
        sIdle += (wv[1] - wv[0]) - B;
        sHid += K + UM - B;
    }
    E = warp_max64(E);
    sU = warp_sum64(sU);
    sW = warp_sum64(sW);
    sP = warp_sum64(sP);
    maxUW = warp_max64(maxUW);
    not_tiled = __reduce_or_sync(0xFFFFFFFFu, not_tiled);
    sK = warp_sum64(sK);
    maxK = warp_max64(maxK);
    maxB = warp_max64(maxB);
    sM = warp_sum64(sM);
    sIdle = warp_sum64(sIdle);
    sHid = warp_sum64(sHid);
    if (lane != 0) return;

    uint32_t fl = 0;
    if (not_tiled) fl |= 0x2u;
    const uint32_t st = *t.status;
    if (st & (ST_BAD_END | ST_BAD_KIND)) fl |= 0x100u;
    if (st & ST_UNSORTED) fl |= 0x200u;
    if (st & ST_TIMEOUT) fl |= 0x400u;
    MetricsOut o;
    o.trace_id = t.trace_id;
    o.region = r;
    o.n_ranks = t.n;
    o.m_devices = t.m;
    o.elapsed_ns = E;
    o.sum_useful = sU;
    o.sum_offload = sW;
    o.sum_mpi = sP;
    o.max_useful_offload = maxUW;
    o.sum_kernel = sK;
    o.max_kernel = maxK;
    o.max_busy = maxB;
    o.sum_mem = sM;
    o.sum_idle = sIdle;
    o.sum_hidden_mem = sHid;
    o.flags = fl;
    form_ratios(o);
    *job.out = o;
}

// ------------------------------------------------------------- thread tree
//
// Host tree with threads.  The paper's host tree has one set of intervals per
// MPI rank; here every thread is a host unit of the trace and proc_off groups
// the units into processes.  One CTA per (trace, region).  A warp takes one
// process at a time, its lanes over the process's threads, and reduces their
// busy time B = U + W to its maximum M_i (the busiest thread) together with
// the sums of U and W and the largest U + W + MPI.  The CTA then reduces
//   E = max over threads (U + W + MPI), sum U, sum W, sum_i T_i M_i, max_i M_i
// and forms, in FP64 in this order (0/0 reads 1, E = 0 gives EMPTY with
// every ratio 1):
//   PE = sum U / (E nT)          MPI PE = sum T M / (E nT)
//   MPI LB = sum T M / (nT max M)   MPI CE = max M / E
//   thread LB = sum B / sum T M     OE = sum U / sum B
// With one thread per process these are the Eqs. 6-8 values of finalize.
// The six ratios from a thread record's aggregates (o.flags holds the status
// bits on entry; EMPTY is set here): nT = o.n_threads.
__device__ __forceinline__ void form_thread_ratios(ThreadOut& o) {
    const int64_t E = o.elapsed_ns, nT = o.n_threads;
    const int64_t sU = o.sum_useful, sW = o.sum_offload, sTM = o.sum_busiest, maxM = o.max_busiest;
    if (E == 0) {
        o.flags |= 0x1u;
        o.pe = o.mpi_pe = o.mpi_lb = o.mpi_ce = o.thread_lb = o.oe = 1.0;
        return;
    }
    o.pe = ratio_k(sU, E, nT);
    o.mpi_pe = ratio_k(sTM, E, nT);
    o.mpi_lb = ratio_k(sTM, nT, maxM);
    o.mpi_ce = ratio(maxM, E);
    o.thread_lb = ratio(sU + sW, sTM);
    o.oe = ratio(sU, sU + sW);
}

__global__ void __launch_bounds__(256) thread_tree_kernel(const ThreadJob* __restrict__ jobs) {
    __shared__ long long sh[32];
    const ThreadJob job = jobs[blockIdx.x];
    const TraceDev t = *job.t;
    const uint32_t r = job.region, R = t.R;
    const int lane = threadIdx.x & 31;
    const uint32_t nw = blockDim.x >> 5;
    auto add = [](long long a, long long b) { return a + b; };
    auto mx = [](long long a, long long b) { return a > b ? a : b; };

    long long E = 0, sU = 0, sW = 0, sTM = 0, maxM = 0;
    for (uint32_t i = threadIdx.x >> 5; i < job.n_procs; i += nw) {
        const uint32_t u0 = job.proc_off[i], u1 = job.proc_off[i + 1];
        int64_t e = 0, pu = 0, pw = 0, m = 0;
        for (uint32_t u = u0 + lane; u < u1; u += 32) {
            const int64_t* h = t.hsum + (static_cast<uint64_t>(u) * R + r) * 3;
            const int64_t U = h[0], W = h[1], P = h[2];
            e = max64(e, U + W + P);
            pu += U;
            pw += W;
            m = max64(m, U + W);
        }
        e = warp_max64(e);
        pu = warp_sum64(pu);
        pw = warp_sum64(pw);
        m = warp_max64(m);
        if (lane == 0) {
            E = mx(E, e);
            sU += pu;
            sW += pw;
            sTM += static_cast<long long>(u1 - u0) * m;
            maxM = mx(maxM, m);
        }
    }
    E = block_reduce<long long>(E, mx, sh);
    sU = block_reduce<long long>(sU, add, sh);
    sW = block_reduce<long long>(sW, add, sh);
    sTM = block_reduce<long long>(sTM, add, sh);
    maxM = block_reduce<long long>(maxM, mx, sh);
    if (threadIdx.x != 0) return;

    const int64_t nT = job.proc_off[job.n_procs];
    uint32_t fl = 0;
    const uint32_t st = *t.status;
    if (st & (ST_BAD_END | ST_BAD_KIND)) fl |= 0x100u;
    if (st & ST_UNSORTED) fl |= 0x200u;
    if (st & ST_TIMEOUT) fl |= 0x400u;
    ThreadOut o;
    o.trace_id = t.trace_id;
    o.region = r;
    o.n_procs = job.n_procs;
    o.n_threads = static_cast<uint32_t>(nT);
    o.elapsed_ns = E;
    o.sum_useful = sU;
    o.sum_offload = sW;
    o.sum_busiest = sTM;
    o.max_busiest = maxM;
    o.flags = fl;
    form_thread_ratios(o);
    *job.out = o;
}

// Thread-tree aggregates of disjoint shards of a trace (whole processes with
// their threads) combine exactly: E and max M by max, the sums and the
// process and thread counts by addition, the status flags by or; the ratios
// are then formed by the same code.
__global__ void __launch_bounds__(256) thread_combine_kernel(const ThreadOut* __restrict__ parts, uint32_t n_parts,
                                                             ThreadOut* __restrict__ out) {
    __shared__ long long sh[32];
    auto add = [](long long a, long long b) { return a + b; };
    auto mx = [](long long a, long long b) { return a > b ? a : b; };
    auto bor = [](long long a, long long b) { return a | b; };
    long long E = 0, sU = 0, sW = 0, sTM = 0, maxM = 0, np = 0, nt = 0, fl = 0;
    for (uint32_t k = threadIdx.x; k < n_parts; k += blockDim.x) {
        const ThreadOut& p = parts[k];
        E = mx(E, p.elapsed_ns);
        sU += p.sum_useful;
        sW += p.sum_offload;
        sTM += p.sum_busiest;
        maxM = mx(maxM, p.max_busiest);
        np += p.n_procs;
        nt += p.n_threads;
        fl |= p.flags & 0x700u;   // status bits; EMPTY is recomputed
    }
    E = block_reduce<long long>(E, mx, sh);
    sU = block_reduce<long long>(sU, add, sh);
    sW = block_reduce<long long>(sW, add, sh);
    sTM = block_reduce<long long>(sTM, add, sh);
    maxM = block_reduce<long long>(maxM, mx, sh);
    np = block_reduce<long long>(np, add, sh);
    nt = block_reduce<long long>(nt, add, sh);
    fl = block_reduce<long long>(fl, bor, sh);
    if (threadIdx.x != 0) return;
    ThreadOut o;
    o.trace_id = parts[0].trace_id;
    o.region = parts[0].region;
    o.n_procs = static_cast<uint32_t>(np);
    o.n_threads = static_cast<uint32_t>(nt);
    o.elapsed_ns = E;
    o.sum_useful = sU;
    o.sum_offload = sW;
    o.sum_busiest = sTM;
    o.max_busiest = maxM;
    o.flags = static_cast<uint32_t>(fl);
    form_thread_ratios(o);
    *out = o;
}

cudaError_t launch_thread_combine(const ThreadOut* parts, uint32_t n_parts, ThreadOut* out, cudaStream_t stream) {
    if (n_parts == 0) return cudaSuccess;
    thread_combine_kernel<<<1, 256, 0, stream>>>(parts, n_parts, out);
    return cudaGetLastError();
}

cudaError_t launch_thread_tree(const ThreadJob* jobs, uint32_t n_jobs, cudaStream_t stream) {
    if (n_jobs == 0) return cudaSuccess;
    thread_tree_kernel<<<n_jobs, 256, 0, stream>>>(jobs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- combine
//
// Aggregates of one region computed on disjoint shards of a trace (whole
// ranks with their devices) combine exactly: E and the maxima by max, the
// sums and the unit counts by addition, the status bits by or.  One CTA
// reduces the shard records and forms the ratios with the same code as the
// single-shard finalize.
__global__ void __launch_bounds__(256) combine_kernel(const MetricsOut* __restrict__ parts, uint32_t n_parts,
                                                      MetricsOut* __restrict__ out) {
    __shared__ long long sh[32];
    auto add = [](long long a, long long b) { return a + b; };
    auto mx = [](long long a, long long b) { return a > b ? a : b; };
    auto bor = [](long long a, long long b) { return a | b; };
    long long E = 0, sU = 0, sW = 0, sP = 0, maxUW = 0, sK = 0, maxK = 0, maxB = 0, sM = 0, sIdle = 0, sHid = 0;
    long long n = 0, m = 0, fl = 0;
    for (uint32_t k = threadIdx.x; k < n_parts; k += blockDim.x) {
        const MetricsOut& p = parts[k];
        E = mx(E, p.elapsed_ns);
        sU += p.sum_useful;
        sW += p.sum_offload;
        sP += p.sum_mpi;
        maxUW = mx(maxUW, p.max_useful_offload);
        sK += p.sum_kernel;
        maxK = mx(maxK, p.max_kernel);
        maxB = mx(maxB, p.max_busy);
        sM += p.sum_mem;
        sIdle += p.sum_idle;
        sHid += p.sum_hidden_mem;
        n += p.n_ranks;
        m += p.m_devices;
        fl |= p.flags & 0x702u;   // status bits and HOST_NOT_TILED; EMPTY / NO_DEVICES are recomputed
    }
    E = block_reduce<long long>(E, mx, sh);
    sU = block_reduce<long long>(sU, add, sh);
    sW = block_reduce<long long>(sW, add, sh);
    sP = block_reduce<long long>(sP, add, sh);
    maxUW = block_reduce<long long>(maxUW, mx, sh);
    sK = block_reduce<long long>(sK, add, sh);
    maxK = block_reduce<long long>(maxK, mx, sh);
    maxB = block_reduce<long long>(maxB, mx, sh);
    sM = block_reduce<long long>(sM, add, sh);
    sIdle = block_reduce<long long>(sIdle, add, sh);
    sHid = block_reduce<long long>(sHid, add, sh);
    n = block_reduce<long long>(n, add, sh);
    m = block_reduce<long long>(m, add, sh);
    fl = block_reduce<long long>(fl, bor, sh);
    if (threadIdx.x != 0) return;
    MetricsOut o;
    o.trace_id = parts[0].trace_id;
    o.region = parts[0].region;
    o.n_ranks = static_cast<uint32_t>(n);
    o.m_devices = static_cast<uint32_t>(m);
    o.elapsed_ns = E;
    o.sum_useful = sU;
    o.sum_offload = sW;
    o.sum_mpi = sP;
    o.max_useful_offload = maxUW;
    o.sum_kernel = sK;
    o.max_kernel = maxK;
    o.max_busy = maxB;
    o.sum_mem = sM;
    o.sum_idle = sIdle;
    o.sum_hidden_mem = sHid;
    o.flags = static_cast<uint32_t>(fl);
    form_ratios(o);
    *out = o;
}

// ------------------------------------------------------------ scalability
//
// POP's second branch across runs (TALP leaves it to the user, Sec. 3.3):
// per run, against the reference run, speedup E_ref / E_r, computation
// scalability from the useful (host) and kernel (device) sums -- strong:
// sum_ref / sum_r; weak: (sum_ref * units_r) / (sum_r * units_ref) -- and
// global efficiency = parallel efficiency x computation scalability.  FP64
// in the order written, round to nearest; a zero denominator reads 1.
__device__ __forceinline__ double ratio_scaled(int64_t num, int64_t k_num, int64_t den, int64_t k_den) {
    const double d = __dmul_rn(__ll2double_rn(den), __ll2double_rn(k_den));
    if (d == 0.0) return 1.0;
    return __ddiv_rn(__dmul_rn(__ll2double_rn(num), __ll2double_rn(k_num)), d);
}

__global__ void scalability_kernel(const MetricsOut* __restrict__ runs, uint32_t n_runs, uint32_t ref, int weak,
                                   ScaleOut* __restrict__ out) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_runs) return;
    const MetricsOut& b = runs[ref];
    const MetricsOut& x = runs[r];
    ScaleOut o;
    o.trace_id = x.trace_id;
    o.region = x.region;
    o.flags = x.flags & 0x707u;
    o.n_ranks = x.n_ranks;
    o.m_devices = x.m_devices;
    o.speedup = ratio(b.elapsed_ns, x.elapsed_ns);
    o.host_comp_scal = weak ? ratio_scaled(b.sum_useful, x.n_ranks, x.sum_useful, b.n_ranks)
                            : ratio(b.sum_useful, x.sum_useful);
    o.host_global_eff = __dmul_rn(x.host_pe, o.host_comp_scal);
    o.dev_comp_scal = weak ? ratio_scaled(b.sum_kernel, x.m_devices, x.sum_kernel, b.m_devices)
                           : ratio(b.sum_kernel, x.sum_kernel);
    o.dev_global_eff = __dmul_rn(x.dev_pe, o.dev_comp_scal);
    out[r] = o;
}

cudaError_t launch_scalability(const MetricsOut* runs, uint32_t n_runs, uint32_t ref, int weak, ScaleOut* out,
                               cudaStream_t stream) {
    if (n_runs == 0) return cudaSuccess;
    scalability_kernel<<<(n_runs + 127) / 128, 128, 0, stream>>>(runs, n_runs, ref, weak, out);
    return cudaGetLastError();
}

cudaError_t launch_combine(const MetricsOut* parts, uint32_t n_parts, MetricsOut* out, cudaStream_t stream) {
    if (n_parts == 0) return cudaSuccess;
    combine_kernel<<<1, 256, 0, stream>>>(parts, n_parts, out);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeJob* jobs, uint32_t n_jobs, cudaStream_t stream) {
    if (n_jobs == 0) return cudaSuccess;
    finalize_kernel<<<(n_jobs + kFinWarps - 1) / kFinWarps, 32 * kFinWarps, 0, stream>>>(jobs, n_jobs);
    return cudaGetLastError();
}

}  // namespace talp
