/*
 * CPU oracle for the extended POP efficiency metrics (host and device trees).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes; it is used by the tests, by the
 * smoke check and by the benchmark's CPU-baseline leg, never by the product
 * path.  It shares no code, header, table or constant with the CUDA library.
 *
 * Paper: "Hardware-Agnostic and Insightful Efficiency Metrics for Accelerated
 * Systems" (arXiv 2603.26576).
 *   - POP model, Sec. 3.3: elapsed time E (Eq. 1), useful sums (Eq. 2).
 *   - Host tree, Sec. 4.1: three host states useful / device offloading / MPI;
 *     PE_host (Eq. 6), MPI_PE_host (Eq. 7) whose load-balance and
 *     communication children treat offloading as useful, OE_host (Eq. 8).
 *   - Device tree, Sec. 4.1: kernel / memory operations / idle per device,
 *     overlap counted as computation; PE (Eq. 9), LB (Eq. 10), CE (Eq. 11),
 *     OE (Eq. 12).
 *   - Post-processing, Sec. 4.2: kernel records merged across streams into a
 *     union; memory records merged and the parts under kernels removed; the
 *     uncovered rest is idle.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - intervals are half open [start, end) in int64 ns; end == start adds 0;
 *   - a region is a per-rank window [a_i, b_i); every host interval of rank i
 *     and every record of a device owned by rank i is clipped to it;
 *   - E = max_i (U_i + W_i + MPI_i), the not-useful set being offload + MPI;
 *     the device metrics use the same E;
 *   - a ratio whose denominator is 0 is 1 (no loss attributable to that
 *     factor); when E == 0 every ratio is 1 and the EMPTY flag is set;
 *   - ratio order in FP64: (double)num / ((double)k * (double)den) for the
 *     forms with n or m in the denominator, (double)num / (double)den else.
 *
 * The host tree with threads at the end is a variant the paper does not
 * define (one thread per process gives back the paper's tree exactly).
 *
 * Parity is pinned (tests/test_oracle_pins.py) by brute-force per-ns tick
 * counting, closed forms, invariants, and the paper's synthetic-benchmark
 * tables; no function here is "parity unpinned".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t s, e;
} ivl_t;

static int cmp_start(const void *pa, const void *pb) {
    const ivl_t *a = (const ivl_t *)pa, *b = (const ivl_t *)pb;
    if (a->s < b->s) return -1;
    if (a->s > b->s) return 1;
    return 0;
}

static int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

/* |union of the given intervals|: sort by start, then one linear merge. */
static int64_t union_length(ivl_t *v, size_t k) {
    if (k == 0) return 0;
    qsort(v, k, sizeof(ivl_t), cmp_start);
    int64_t total = 0;
    int64_t cs = v[0].s, ce = v[0].e;
    for (size_t j = 1; j < k; ++j) {
        if (v[j].s > ce) {          /* disjoint: close the current run */
            total += ce - cs;
            cs = v[j].s;
            ce = v[j].e;
        } else if (v[j].e > ce) {   /* overlapping or touching: extend */
            ce = v[j].e;
        }
    }
    total += ce - cs;
    return total;
}

/*
 * Record checks (the library reports invalid input instead of computing):
 * end < start, a device kind above 4, a host state above 2.
 * Returns 0 when the trace is valid, else a bit set: 1 = host end < start,
 * 2 = bad host state, 4 = device end < start, 8 = bad device kind.
 */
int oracle_validate(uint64_t n_host, const int64_t *host_se, const uint8_t *host_state,
                    uint64_t n_dev, const int64_t *dev_se, const uint8_t *dev_tag) {
    int bad = 0;
    for (uint64_t j = 0; j < n_host; ++j) {
        if (host_se[2 * j + 1] < host_se[2 * j]) bad |= 1;
        if (host_state[j] > 2) bad |= 2;
    }
    for (uint64_t j = 0; j < n_dev; ++j) {
        if (dev_se[2 * j + 1] < dev_se[2 * j]) bad |= 4;
        if ((dev_tag[j] >> 5) > 4) bad |= 8;
    }
    return bad;
}

/*
 * Host state sums of one region (Sec. 4.1 three host states; Eq. 2 applied
 * to each state).  For every rank i and state q in {useful, offload, MPI}:
 *   out[i][q] = sum over host intervals h of rank i with state q of
 *               |[max(s_h, a_i), min(e_h, b_i))|  (0 when empty).
 * win is [n][2] = [a_i, b_i) for this region.
 */
void oracle_host_sums(uint32_t n_ranks, const int64_t *host_se, const uint8_t *host_state,
                      const uint64_t *host_off, const int64_t *win, int64_t *out) {
    for (uint32_t i = 0; i < n_ranks; ++i) {
        int64_t a = win[2 * i], b = win[2 * i + 1];
        int64_t acc[3] = {0, 0, 0};
        for (uint64_t j = host_off[i]; j < host_off[i + 1]; ++j) {
            int64_t lo = max64(host_se[2 * j], a);
            int64_t hi = min64(host_se[2 * j + 1], b);
            if (hi > lo) acc[host_state[j]] += hi - lo;
        }
        out[3 * i + 0] = acc[0];
        out[3 * i + 1] = acc[1];
        out[3 * i + 2] = acc[2];
    }
}

/*
 * Device flattening of one region (Sec. 4.1 device states, Sec. 4.2
 * post-processing).  Devices are numbered rank-major: the first
 * devices_per_rank[0] belong to rank 0, and so on.  For device g of rank i
 * the records are clipped to [a_i, b_i) and then
 *   out[g][0] = |union of kernel records|            (D_K, kernel time)
 *   out[g][1] = |union of memory-operation records|   (all transfer time)
 *   out[g][2] = |union of all records|                (busy time B)
 * Memory operations are kinds 1..4 (H2D, D2H, D2D, memset); streams are not
 * distinguished.  The caller derives D_M = B - D_K (transfers not hidden by
 * kernels) and idle = (b_i - a_i) - B.
 * Returns 0, or -1 when memory for the scratch copy cannot be had.
 */
int oracle_device_unions(uint32_t n_ranks, const uint32_t *devices_per_rank, const int64_t *dev_se,
                         const uint8_t *dev_tag, const uint64_t *dev_off, const int64_t *win,
                         int64_t *out) {
    uint32_t g = 0;
    for (uint32_t i = 0; i < n_ranks; ++i) {
        int64_t a = win[2 * i], b = win[2 * i + 1];
        for (uint32_t d = 0; d < devices_per_rank[i]; ++d, ++g) {
            uint64_t lo_idx = dev_off[g], hi_idx = dev_off[g + 1];
            size_t n = (size_t)(hi_idx - lo_idx);
            ivl_t *kv = (ivl_t *)malloc((n ? n : 1) * sizeof(ivl_t));
            ivl_t *mv = (ivl_t *)malloc((n ? n : 1) * sizeof(ivl_t));
            ivl_t *av = (ivl_t *)malloc((n ? n : 1) * sizeof(ivl_t));
            if (!kv || !mv || !av) {
                free(kv); free(mv); free(av);
                return -1;
            }
            size_t nk = 0, nm = 0, na = 0;
            for (uint64_t j = lo_idx; j < hi_idx; ++j) {
                int64_t s = max64(dev_se[2 * j], a);
                int64_t e = min64(dev_se[2 * j + 1], b);
                if (e <= s) continue;
                ivl_t x = {s, e};
                if ((dev_tag[j] >> 5) == 0) kv[nk++] = x; else mv[nm++] = x;
                av[na++] = x;
            }
            out[3 * g + 0] = union_length(kv, nk);
            out[3 * g + 1] = union_length(mv, nm);
            out[3 * g + 2] = union_length(av, na);
            free(kv); free(mv); free(av);
        }
    }
    return 0;
}

/*
 * Concurrency profile of one region (the per-device occupancy the paper
 * leaves to future work on streams, Sec. 4.1): for device g of rank i, with
 * its records clipped to [a_i, b_i) and c(t) the number of them active at
 * time t (a record [s, e) is active for s <= t < e),
 *   out[g][0][k-1] = |{t : c(t) >= k}|                 for k = 1 .. K,
 *   out[g][1][k-1] = the same over kernel records only.
 * Level 1 is the busy union B (resp. the kernel union D_K).  Computed the
 * plain way: +1 / -1 events at every clipped start / end, sorted by time,
 * and the time between consecutive events added to every level up to the
 * count of active records.
 * Returns 0, or -1 when memory for the events cannot be had.
 */
typedef struct {
    int64_t t;
    int d;
} ev_t;

static int cmp_ev(const void *pa, const void *pb) {
    const ev_t *a = (const ev_t *)pa, *b = (const ev_t *)pb;
    if (a->t < b->t) return -1;
    if (a->t > b->t) return 1;
    return 0;
}

static void level_times(ev_t *ev, size_t n, uint32_t K, int64_t *out) {
    for (uint32_t k = 0; k < K; ++k) out[k] = 0;
    if (n == 0) return;
    qsort(ev, n, sizeof(ev_t), cmp_ev);
    int64_t c = 0;
    for (size_t j = 0; j + 1 < n; ++j) {
        c += ev[j].d;
        const int64_t dt = ev[j + 1].t - ev[j].t;
        for (int64_t k = 1; k <= c && k <= (int64_t)K; ++k) out[k - 1] += dt;
    }
}

int oracle_concurrency(uint32_t n_ranks, const uint32_t *devices_per_rank, const int64_t *dev_se,
                       const uint8_t *dev_tag, const uint64_t *dev_off, const int64_t *win, uint32_t K,
                       int64_t *out) {
    uint32_t g = 0;
    for (uint32_t i = 0; i < n_ranks; ++i) {
        int64_t a = win[2 * i], b = win[2 * i + 1];
        for (uint32_t d = 0; d < devices_per_rank[i]; ++d, ++g) {
            uint64_t lo_idx = dev_off[g], hi_idx = dev_off[g + 1];
            size_t n = (size_t)(hi_idx - lo_idx);
            ev_t *ea = (ev_t *)malloc((2 * n + 1) * sizeof(ev_t));
            ev_t *ek = (ev_t *)malloc((2 * n + 1) * sizeof(ev_t));
            if (!ea || !ek) {
                free(ea); free(ek);
                return -1;
            }
            size_t na = 0, nk = 0;
            for (uint64_t j = lo_idx; j < hi_idx; ++j) {
                int64_t s = max64(dev_se[2 * j], a);
                int64_t e = min64(dev_se[2 * j + 1], b);
                if (e <= s) continue;
                ea[na].t = s; ea[na++].d = 1;
                ea[na].t = e; ea[na++].d = -1;
                if ((dev_tag[j] >> 5) == 0) {
                    ek[nk].t = s; ek[nk++].d = 1;
                    ek[nk].t = e; ek[nk++].d = -1;
                }
            }
            level_times(ea, na, K, out + (size_t)g * 2 * K);
            level_times(ek, nk, K, out + (size_t)g * 2 * K + K);
            free(ea); free(ek);
        }
    }
    return 0;
}

/* num / (k * den) with the 0/0 := 1 reading. */
static double ratio_k(int64_t num, int64_t k, int64_t den) {
    if (k == 0 || den == 0) return 1.0;
    double dk = (double)k, dd = (double)den;
    double prod = dk * dd;
    return (double)num / prod;
}

static double ratio(int64_t num, int64_t den) {
    if (den == 0) return 1.0;
    return (double)num / (double)den;
}

/*
 * Metrics of one region from the per-rank and per-device sums.
 *   host_sums [n][3] from oracle_host_sums, dev_unions [m][3] from
 *   oracle_device_unions, win [n][2] the region's windows.
 * iout[11]: E, sum U, sum W, sum MPI, max(U+W), sum D_K, max D_K,
 *           max(D_K + D_M), sum D_M, sum idle, sum hidden transfer.
 * dout[9] : PE_host (Eq. 6), MPI_PE_host (Eq. 7), its LB and CE (Eqs. 4-5
 *           with offloading counted as useful), OE_host (Eq. 8), PE_dev (Eq. 9),
 *           LB_dev (Eq. 10), CE_dev (Eq. 11), OE_dev (Eq. 12).
 * *flags  : 1 = EMPTY (E == 0), 2 = HOST_NOT_TILED (some rank's host sums
 *           differ from its window length), 4 = NO_DEVICES (m == 0: the
 *           device ratios are reported as 1).
 */
void oracle_metrics(uint32_t n_ranks, const uint32_t *devices_per_rank, const int64_t *host_sums,
                    const int64_t *dev_unions, const int64_t *win, int64_t *iout, double *dout,
                    uint32_t *flags) {
    uint32_t m = 0;
    for (uint32_t i = 0; i < n_ranks; ++i) m += devices_per_rank[i];
    uint32_t fl = 0;

    /* host: Eq. 1 with the not-useful set = offload + MPI */
    int64_t E = 0, sU = 0, sW = 0, sMPI = 0, maxUW = 0;
    for (uint32_t i = 0; i < n_ranks; ++i) {
        int64_t U = host_sums[3 * i + 0], W = host_sums[3 * i + 1], P = host_sums[3 * i + 2];
        E = max64(E, U + W + P);
        sU += U;
        sW += W;
        sMPI += P;
        maxUW = max64(maxUW, U + W);
        if (U + W + P != win[2 * i + 1] - win[2 * i]) fl |= 2;
    }

    /* device: per device D_K, D_M = B - D_K, idle = window - B */
    int64_t sK = 0, maxK = 0, maxB = 0, sM = 0, sIdle = 0, sHidden = 0;
    uint32_t g = 0;
    for (uint32_t i = 0; i < n_ranks; ++i) {
        int64_t len = win[2 * i + 1] - win[2 * i];
        for (uint32_t d = 0; d < devices_per_rank[i]; ++d, ++g) {
            int64_t K = dev_unions[3 * g + 0];
            int64_t UM = dev_unions[3 * g + 1];
            int64_t B = dev_unions[3 * g + 2];
            int64_t DM = B - K;
            sK += K;
            maxK = max64(maxK, K);
            maxB = max64(maxB, K + DM);
            sM += DM;
            sIdle += len - B;
            sHidden += K + UM - B;
        }
    }

    iout[0] = E; iout[1] = sU; iout[2] = sW; iout[3] = sMPI; iout[4] = maxUW;
    iout[5] = sK; iout[6] = maxK; iout[7] = maxB; iout[8] = sM; iout[9] = sIdle; iout[10] = sHidden;

    if (E == 0) {
        fl |= 1;
        for (int q = 0; q < 9; ++q) dout[q] = 1.0;
        if (m == 0) fl |= 4;
        *flags = fl;
        return;
    }
    dout[0] = ratio_k(sU, E, (int64_t)n_ranks);           /* Eq. 6 */
    dout[1] = ratio_k(sU + sW, E, (int64_t)n_ranks);      /* Eq. 7 */
    dout[2] = ratio_k(sU + sW, (int64_t)n_ranks, maxUW);  /* Eq. 4, U+W as useful */
    dout[3] = ratio(maxUW, E);                            /* Eq. 5, U+W as useful */
    dout[4] = ratio(sU, sU + sW);                         /* Eq. 8 */
    if (m == 0) {                                         /* no device tree */
        fl |= 4;
        for (int q = 5; q < 9; ++q) dout[q] = 1.0;
    } else {
        dout[5] = ratio_k(sK, E, (int64_t)m);             /* Eq. 9 */
        dout[6] = ratio_k(sK, (int64_t)m, maxK);          /* Eq. 10 */
        dout[7] = ratio(maxK, maxB);                      /* Eq. 11 */
        dout[8] = ratio(maxB, E);                         /* Eq. 12 */
    }
    *flags = fl;
}

/*
 * Scalability across runs (POP's second branch, which TALP leaves to the
 * user across several runs, Sec. 3.3): the region metrics of n_runs runs of
 * one application at different scales against the reference run `ref`.
 * For run r (iruns[r] = {E, sum U, sum D_K}, units[r] = {n, m}, pe[r] =
 * {PE_host, PE_dev} as computed above):
 *   out[r][0] = speedup            E_ref / E_r
 *   out[r][1] = host comp. scal.   strong: sumU_ref / sumU_r
 *                                  weak:   (sumU_ref * n_r) / (sumU_r * n_ref)
 *   out[r][2] = host global eff.   PE_host_r * out[r][1]
 *   out[r][3] = device comp. scal. the same with sum D_K and m
 *   out[r][4] = device global eff. PE_dev_r * out[r][3]
 * FP64, round to nearest, the order as written; a zero denominator reads 1.
 */
static double ratio_scaled(int64_t num, int64_t k_num, int64_t den, int64_t k_den) {
    double d = (double)den * (double)k_den;
    if (d == 0.0) return 1.0;
    return ((double)num * (double)k_num) / d;
}

void oracle_scalability(uint32_t n_runs, const int64_t *iruns, const uint32_t *units, const double *pe,
                        uint32_t ref, int weak, double *out) {
    const int64_t E0 = iruns[3 * ref], U0 = iruns[3 * ref + 1], K0 = iruns[3 * ref + 2];
    const int64_t n0 = units[2 * ref], m0 = units[2 * ref + 1];
    for (uint32_t r = 0; r < n_runs; ++r) {
        const int64_t E = iruns[3 * r], U = iruns[3 * r + 1], Kd = iruns[3 * r + 2];
        const int64_t n = units[2 * r], m = units[2 * r + 1];
        double *o = out + 5 * r;
        o[0] = ratio(E0, E);
        o[1] = weak ? ratio_scaled(U0, n, U, n0) : ratio(U0, U);
        o[2] = pe[2 * r] * o[1];
        o[3] = weak ? ratio_scaled(K0, m, Kd, m0) : ratio(K0, Kd);
        o[4] = pe[2 * r + 1] * o[3];
    }
}

/*
 * Host tree with threads.  The paper's host tree (Sec. 4.1, Eqs. 6-8) has one
 * set of host intervals per MPI rank and no thread level; this variant gives
 * every thread of a process its own useful / offload / MPI intervals (one
 * host unit per thread) and adds one factor for how evenly the threads of a
 * process are busy.  Process i owns the host units proc_off[i] ..
 * proc_off[i+1]-1, T_i >= 1 of them.  Per thread, from host_sums (as
 * oracle_host_sums returns them for the units): B = U + W (busy).  Then
 *   M_i = max over the threads of process i of B   (its busiest thread)
 *   nT  = sum_i T_i
 *   E   = max over all threads of (U + W + MPI)     (Eq. 1 over threads)
 *   PE        = sum U / (E nT)                      (Eq. 6 over threads)
 *   MPI PE    = sum_i T_i M_i / (E nT)              (Eq. 7 with the busiest thread
 *                                                    standing for its process)
 *     MPI LB  = sum_i T_i M_i / (nT max_i M_i)
 *     MPI CE  = max_i M_i / E
 *   thread LB = sum B / sum_i T_i M_i               (Eq. 10's average-over-max form,
 *                                                    inside each process)
 *   OE        = sum U / sum B                       (Eq. 8 over threads)
 * so PE = MPI PE x thread LB x OE and MPI PE = MPI LB x MPI CE; with one
 * thread per process every value equals the paper's host tree (thread LB = 1).
 * FP64 in the order written with ratio_k / ratio above; 0/0 reads 1.
 * iout[6]: E, sum U, sum W, sum_i T_i M_i, max_i M_i, nT.
 * dout[6]: PE, MPI PE, MPI LB, MPI CE, thread LB, OE.
 * *flags : 1 = EMPTY (E == 0, every ratio 1).
 */
void oracle_thread_metrics(uint32_t n_procs, const uint32_t *proc_off, const int64_t *host_sums,
                           int64_t *iout, double *dout, uint32_t *flags) {
    int64_t E = 0, sU = 0, sW = 0, sTM = 0, maxM = 0, nT = 0;
    for (uint32_t i = 0; i < n_procs; ++i) {
        const int64_t T = (int64_t)proc_off[i + 1] - (int64_t)proc_off[i];
        int64_t M = 0;
        for (uint32_t u = proc_off[i]; u < proc_off[i + 1]; ++u) {
            const int64_t U = host_sums[3 * u + 0], W = host_sums[3 * u + 1], P = host_sums[3 * u + 2];
            E = max64(E, U + W + P);
            sU += U;
            sW += W;
            M = max64(M, U + W);
        }
        sTM += T * M;
        maxM = max64(maxM, M);
        nT += T;
    }
    iout[0] = E; iout[1] = sU; iout[2] = sW; iout[3] = sTM; iout[4] = maxM; iout[5] = nT;
    *flags = 0;
    if (E == 0) {
        *flags = 1;
        for (int q = 0; q < 6; ++q) dout[q] = 1.0;
        return;
    }
    dout[0] = ratio_k(sU, E, nT);
    dout[1] = ratio_k(sTM, E, nT);
    dout[2] = ratio_k(sTM, nT, maxM);
    dout[3] = ratio(maxM, E);
    dout[4] = ratio(sU + sW, sTM);
    dout[5] = ratio(sU, sU + sW);
}
