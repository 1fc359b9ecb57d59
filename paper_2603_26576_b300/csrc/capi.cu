// Host engine behind the C ABI: trace table, HBM admission, host-pointer
// staging, segment tables, the launch sequence (prep -> sweep -> fix-up ->
// [sort -> re-sweep -> fix-up] -> [finalize]), the result calls, and
// reusable plans captured as CUDA graphs with an autotuned sweep shape.
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/talp_gpu.h"
#include "engine.h"
#include "kernels.h"

using namespace talp;

static_assert(sizeof(MetricsOut) == sizeof(talp_gpu_metrics), "metrics layout");
static_assert(offsetof(MetricsOut, elapsed_ns) == offsetof(talp_gpu_metrics, elapsed_ns), "metrics layout");
static_assert(offsetof(MetricsOut, host_pe) == offsetof(talp_gpu_metrics, host_pe), "metrics layout");
static_assert(offsetof(MetricsOut, dev_oe) == offsetof(talp_gpu_metrics, dev_oe), "metrics layout");
static_assert(sizeof(SegDesc) == 80, "segment descriptor layout");

namespace {

thread_local std::string g_last_error;

talp_gpu_status fail(talp_gpu_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

talp_gpu_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return TALP_GPU_ECUDA;
}

#define TALP_CUDA(call)                                     \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

#define TALP_TRY(call)                                      \
    do {                                                    \
        talp_gpu_status s_ = (call);                        \
        if (s_ != TALP_GPU_OK) return s_;                   \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Per-trace device state: partial sums, windows, running carries.
struct RawHold;   // held-back raw records of a trace

struct TraceState {
    uint64_t id = 0;
    uint32_t n = 0, m = 0, R = 0;
    std::vector<uint32_t> dpr;
    void* dmem = nullptr;
    size_t dbytes = 0;
    int64_t* hsum = nullptr;       // [n][R][3]
    int64_t* dsum = nullptr;       // [m][R][3]
    int64_t* hwin = nullptr;       // [n][R][2]
    int64_t* dev_rank = nullptr;   // [m]
    int64_t* carry[2] = {nullptr, nullptr};  // [m][3] each
    uint32_t* status = nullptr;    // one word (+ padding)
    TraceDev* tdev = nullptr;
    int cur = 0;
    int plan_refs = 0;             // plans whose graphs point at this state
};

size_t trace_bytes(uint32_t n, uint32_t m, uint32_t R) {
    size_t b = 0;
    b += align_up(sizeof(int64_t) * n * R * 3, 256);
    b += align_up(sizeof(int64_t) * m * R * 3, 256);
    b += align_up(sizeof(int64_t) * n * R * 2, 256);
    b += align_up(sizeof(int64_t) * (m ? m : 1), 256);
    b += 2 * align_up(sizeof(int64_t) * 3 * (m ? m : 1), 256);
    b += 256;                                         // status
    b += align_up(sizeof(TraceDev), 256);
    return b;
}

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct PinBuf {
    void* p = nullptr;
    size_t cap = 0;
};

// Everything an ingest needs to know before touching memory: sizes, grid,
// and the byte layout of its workspace (upload part first).
struct Tuning {
    int shape = kDefaultSweepShape;
    int tpw = 4;              // minimum tiles per warp (grid sizing of small ingests)
    uint64_t seg_cost = 0;    // phantom records per segment (balances segment switches)
    int spw = 0;              // slices per warp handed out by a ticket (0: one fixed slice per warp)
};

struct Layout {
    int shape = 0, warps = 0, tile = 0, grid = 0, full_grid = 0, tpw = 4, spw = 0;
    uint64_t seg_cost = 0;
    uint32_t rmax = 1, n_wrec = 0, n_wrec_cap = 0;
    uint64_t n_segs = 0, n_records = 0, n_dev_segs = 0;
    uint64_t n_grouped = 0;   // device segments whose runs come from their stream ids
    uint64_t sort_slots = 0, sort_recs = 0, sort_tiles = 0;
    size_t n_backup_words = 0, payload_words = 0, n_jobs_max = 0, n_fin = 0;
    bool sorting = false;
    size_t off_segs = 0, off_start = 0, off_send = 0, off_jobs = 0, off_rest = 0, off_sctl = 0, off_fin = 0,
           off_pay = 0, off_rrend = 0, off_grp = 0;
    uint64_t virt = 0;        // virtual positions (records + phantoms)
    size_t up_bytes = 0;
    size_t off_wrec = 0, off_flags = 0, off_gst = 0, off_bk = 0, off_slist = 0, off_srb = 0, off_stb = 0;
    size_t off_smn = 0, off_smx = 0, off_hist = 0, off_offs = 0, off_rsegs = 0, off_rstart = 0, off_mout = 0;
    size_t off_nruns = 0, off_runs = 0, off_fused = 0, off_known = 0, off_given = 0, off_seen_n = 0, off_seen_pos = 0;
    uint64_t fms_samples = 0, fms_chunks = 0, fms_super = 0;   // table bounds of the fused merge-sweep
    size_t off_fS = 0, off_fsb = 0, off_fcb = 0, off_fpb = 0, off_fscb = 0, off_fsamp = 0, off_fsplit = 0,
           off_fseg = 0, off_fchunk = 0, off_fscagg = 0, off_ffix = 0;
    size_t ws_bytes = 0, stage_bytes = 0, sortbuf_bytes = 0, new_bytes = 0;
    uint32_t nj = 0;
    std::vector<uint64_t> nh, nd;
    std::vector<uint32_t> mm;
};

}  // namespace

void talp::set_last_error(const std::string& msg) { g_last_error = msg; }

// (definitions of the engine.h hooks follow the context struct)

struct talp_gpu_ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;
    size_t held = 0;
    std::unordered_map<uint64_t, TraceState*> traces;
    DevBuf ws;          // segment table, starts, jobs, payload, warp records, flags, sort control
    DevBuf stage;       // host-pointer record staging
    DevBuf sortbuf;     // ping-pong copies of the device segments being sorted
    DevBuf raw;         // raw activity records: staging, lanes, counters
    PinBuf up, down;    // pinned upload / download scratch
    PinBuf upf;         // pinned upload scratch of result calls (their own, so that an ingest
                        // followed by a result call never waits for the ingest's upload)
    cudaEvent_t ev_up = nullptr;      // upload scratch free again
    cudaEvent_t ev_upf = nullptr;     // result-call upload scratch free again
    cudaEvent_t ev_ws = nullptr;      // workspace/staging free again
    cudaEvent_t ev_raw = nullptr;     // raw-record buffer free again
    bool raw_used = false;
    bool ws_used = false;
    Tuning defaults;
    bool shape_forced = false;
    std::unordered_map<uint64_t, Tuning> tune;   // size class -> tuning picked by a plan's autotuner
    cudaStream_t cap_stream = nullptr;                         // stream used for graph capture
    // profiling
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    std::vector<uint64_t> ev_records;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> sort_ev_pending;
    uint64_t kernel_launches = 0;
    int64_t wait_limit = 4000000000LL;   // cycles (~2 s at 2 GHz)
    int dependents = 0;                  // live plans and servers on this context
    std::unordered_map<uint64_t, RawHold*> holds;   // trace id -> held-back raw records
    bool raw_inner = false;              // ingest_events called by ingest_raw
    std::vector<uint8_t> raw_presort;    // with raw_inner: per device of the ingest, known out of order
    const uint64_t* raw_runs = nullptr;  // with raw_inner: per device of the ingest, its lane's known runs
                                         // (device memory, kRunsStride entries each)
};

const TraceDev* talp::trace_device_desc(talp_gpu_ctx* c, uint64_t trace_id, uint32_t* n_regions) {
    auto it = c->traces.find(trace_id);
    if (it == c->traces.end()) return nullptr;
    if (n_regions) *n_regions = it->second->R;
    return it->second->tdev;
}

int talp::ctx_device(talp_gpu_ctx* c) { return c->device; }

void talp::ctx_hold(talp_gpu_ctx* c, int delta) { c->dependents += delta; }

struct talp_gpu_plan {
    talp_gpu_ctx* c = nullptr;
    DevBuf ws, sortbuf;
    PinBuf up;
    Layout L;
    std::vector<TraceState*> ts;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t n_metrics = 0;
    uint64_t launches_per_run = 0;
};

namespace {

talp_gpu_status dev_alloc(talp_gpu_ctx* c, void** p, size_t bytes) {
    if (c->held + bytes > c->budget)
        return fail(TALP_GPU_ENOMEM, "HBM budget exceeded: need " + std::to_string(bytes) + " more bytes, hold " +
                                         std::to_string(c->held) + " of " + std::to_string(c->budget));
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TALP_GPU_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->held += bytes;
    return TALP_GPU_OK;
}

void dev_free(talp_gpu_ctx* c, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    c->held -= bytes;
}

size_t grow_size(size_t need) { return align_up(need + need / 4, 1 << 20); }

talp_gpu_status grow(talp_gpu_ctx* c, DevBuf& b, size_t need) {
    if (b.cap >= need) return TALP_GPU_OK;
    size_t cap = grow_size(need);
    if (b.p) {
        cudaDeviceSynchronize();
        dev_free(c, b.p, b.cap);
        b.p = nullptr;
        b.cap = 0;
    }
    talp_gpu_status st = dev_alloc(c, &b.p, cap);
    if (st != TALP_GPU_OK) return st;
    b.cap = cap;
    return TALP_GPU_OK;
}

talp_gpu_status grow_pinned(PinBuf& b, size_t need) {
    if (b.cap >= need) return TALP_GPU_OK;
    size_t cap = align_up(need + need / 4, 1 << 16);
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
    cudaError_t e = cudaMallocHost(&b.p, cap);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    b.cap = cap;
    return TALP_GPU_OK;
}

cudaEvent_t take_event(talp_gpu_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void free_trace(talp_gpu_ctx* c, TraceState* t) {
    if (!t) return;
    dev_free(c, t->dmem, t->dbytes);
    delete t;
}

talp_gpu_status alloc_trace(talp_gpu_ctx* c, uint64_t id, uint32_t n, const uint32_t* dpr, uint32_t R,
                            TraceState** out) {
    TraceState* t = new TraceState();
    t->id = id;
    t->n = n;
    t->R = R;
    t->dpr.assign(dpr, dpr + n);
    uint64_t m = 0;
    for (uint32_t i = 0; i < n; ++i) m += dpr[i];
    t->m = static_cast<uint32_t>(m);
    t->dbytes = trace_bytes(n, t->m, R);
    talp_gpu_status st = dev_alloc(c, &t->dmem, t->dbytes);
    if (st != TALP_GPU_OK) {
        delete t;
        return st;
    }
    char* p = static_cast<char*>(t->dmem);
    auto take = [&](size_t bytes) {
        char* q = p;
        p += align_up(bytes, 256);
        return q;
    };
    t->hsum = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * n * R * 3));
    t->dsum = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * t->m * R * 3));
    t->hwin = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * n * R * 2));
    t->dev_rank = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * (t->m ? t->m : 1)));
    t->carry[0] = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * 3 * (t->m ? t->m : 1)));
    t->carry[1] = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * 3 * (t->m ? t->m : 1)));
    t->status = reinterpret_cast<uint32_t*>(take(256));
    t->tdev = reinterpret_cast<TraceDev*>(take(sizeof(TraceDev)));
    *out = t;
    return TALP_GPU_OK;
}

bool same_shape(const TraceState* t, const talp_gpu_trace_batch& b) {
    return t->n == b.n_ranks && t->R == b.n_regions &&
           memcmp(t->dpr.data(), b.devices_per_rank, sizeof(uint32_t) * b.n_ranks) == 0;
}

// Host-side checks of one batch header (the records themselves are checked
// on the GPU).
talp_gpu_status check_batch(const talp_gpu_trace_batch& b, uint64_t* n_host, uint64_t* n_dev, uint32_t* m_out) {
    if (b.n_ranks == 0) return fail(TALP_GPU_EINVAL, "n_ranks must be >= 1");
    if (b.n_regions == 0 || b.n_regions > TALP_GPU_MAX_REGIONS)
        return fail(TALP_GPU_EINVAL, "n_regions must be in 1..8");
    if (b.reserved != 0) return fail(TALP_GPU_EINVAL, "reserved must be 0");
    if (b.flags & ~(TALP_GPU_DEVICE_PTRS | TALP_GPU_SORTED_BY_START | TALP_GPU_APPEND | TALP_GPU_NOT_SORTED |
                    TALP_GPU_GROUPED_BY_STREAM))
        return fail(TALP_GPU_EINVAL, "unknown flag bits");
    if ((b.flags & TALP_GPU_SORTED_BY_START) && (b.flags & TALP_GPU_NOT_SORTED))
        return fail(TALP_GPU_EINVAL, "SORTED_BY_START and NOT_SORTED together");
    if ((b.flags & TALP_GPU_GROUPED_BY_STREAM) && (b.flags & (TALP_GPU_SORTED_BY_START | TALP_GPU_NOT_SORTED)))
        return fail(TALP_GPU_EINVAL, "GROUPED_BY_STREAM with SORTED_BY_START or NOT_SORTED");
    if (!b.devices_per_rank || !b.region_window || !b.host_off || !b.dev_off)
        return fail(TALP_GPU_EINVAL, "null header array");
    uint64_t m = 0;
    for (uint32_t i = 0; i < b.n_ranks; ++i) m += b.devices_per_rank[i];
    if (m > 0xFFFFFFF0ull) return fail(TALP_GPU_EINVAL, "too many devices");
    if (b.host_off[0] != 0 || b.dev_off[0] != 0) return fail(TALP_GPU_EINVAL, "offsets must start at 0");
    for (uint32_t i = 0; i < b.n_ranks; ++i)
        if (b.host_off[i + 1] < b.host_off[i]) return fail(TALP_GPU_EINVAL, "host_off not monotone");
    for (uint64_t g = 0; g < m; ++g)
        if (b.dev_off[g + 1] < b.dev_off[g]) return fail(TALP_GPU_EINVAL, "dev_off not monotone");
    for (uint64_t k = 0; k < 2ull * b.n_regions * b.n_ranks; k += 2)
        if (b.region_window[k + 1] < b.region_window[k]) return fail(TALP_GPU_EINVAL, "window end < begin");
    *n_host = b.host_off[b.n_ranks];
    *n_dev = b.dev_off[m];
    *m_out = static_cast<uint32_t>(m);
    if ((*n_host && (!b.host_se || !b.host_state)) || (*n_dev && (!b.dev_se || !b.dev_tag)))
        return fail(TALP_GPU_EINVAL, "null record array");
    if (b.flags & TALP_GPU_DEVICE_PTRS) {
        auto mis = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
        if ((*n_host && (mis(b.host_se) || mis(b.host_state))) || (*n_dev && (mis(b.dev_se) || mis(b.dev_tag))))
            return fail(TALP_GPU_EINVAL, "device record arrays must be 16-byte aligned");
    }
    return TALP_GPU_OK;
}

int ceil_log2(uint64_t x) {
    int b = 0;
    while ((1ull << b) < x && b < 63) ++b;
    return b;
}

// size class of an ingest for the tuning cache
uint64_t size_class(uint64_t records, uint64_t segs, bool sorting) {
    return (static_cast<uint64_t>(ceil_log2(records + 1)) << 16) | (static_cast<uint64_t>(ceil_log2(segs + 1)) << 1) |
           (sorting ? 1u : 0u);
}

// Validation, sizes and workspace layout of an ingest (no side effects).
talp_gpu_status size_ingest(talp_gpu_ctx* c, const talp_gpu_trace_batch* batches, size_t nb, const Tuning& tu,
                            bool with_finalize, Layout& L) {
    const int shape = tu.shape, tpw = tu.tpw;
    L = Layout();
    L.nh.resize(nb);
    L.nd.resize(nb);
    L.mm.resize(nb);
    std::unordered_set<uint64_t> seen;
    for (size_t k = 0; k < nb; ++k) {
        const talp_gpu_trace_batch& b = batches[k];
        TALP_TRY(check_batch(b, &L.nh[k], &L.nd[k], &L.mm[k]));
        if (!seen.insert(b.trace_id).second) return fail(TALP_GPU_EINVAL, "trace id repeated in one call");
        auto it = c->traces.find(b.trace_id);
        if (b.flags & TALP_GPU_APPEND) {
            if (it == c->traces.end()) return fail(TALP_GPU_ENOTFOUND, "APPEND to an unknown trace");
            if (!same_shape(it->second, b)) return fail(TALP_GPU_EINVAL, "APPEND with a different trace shape");
        } else if (it == c->traces.end() || !same_shape(it->second, b)) {
            if (it != c->traces.end() && it->second->plan_refs)
                return fail(TALP_GPU_EBUSY, "a plan uses this trace id with another shape");
            L.new_bytes += trace_bytes(b.n_ranks, L.mm[k], b.n_regions);
        }
        if (!(b.flags & TALP_GPU_DEVICE_PTRS))
            L.stage_bytes += L.nh[k] * 16 + L.nd[k] * 16 + align_up(L.nh[k], 16) + align_up(L.nd[k], 16) + 64;
        L.n_segs += L.mm[k] + b.n_ranks;
        L.n_records += L.nh[k] + L.nd[k];
        L.n_dev_segs += L.mm[k];
        L.rmax = std::max(L.rmax, b.n_regions);
        if (with_finalize) L.n_fin += b.n_regions;
        if (!(b.flags & TALP_GPU_SORTED_BY_START)) {
            L.sort_slots += L.mm[k];
            L.sort_recs += L.nd[k];
            for (uint32_t g = 0; g < L.mm[k]; ++g) {
                const uint64_t nseg = b.dev_off[g + 1] - b.dev_off[g];
                L.sort_tiles += (nseg + sort_tile_records() - 1) / sort_tile_records();
                L.fms_samples += fms_max_samples(nseg);
                L.fms_chunks += fms_max_chunks(nseg);
                L.fms_super += fms_max_super(nseg);
            }
            if ((b.flags & TALP_GPU_APPEND) && L.mm[k]) L.n_backup_words += 3ull * b.n_regions * L.mm[k];
            if (b.flags & TALP_GPU_GROUPED_BY_STREAM) L.n_grouped += L.mm[k];
        }
    }
    if (L.n_segs > 0xFFFFFFF0ull) return fail(TALP_GPU_EINVAL, "too many segments in one call");
    L.sorting = L.sort_slots > 0;
    if (L.sorting) {
        // kernel attribute and grid of the fused merge-sweep, set before any
        // launch sequence is captured
        const cudaError_t e = fms_prepare(c->num_sms);
        if (e != cudaSuccess) return cuda_fail(e, "fused merge-sweep set-up");
    }
    L.sortbuf_bytes = L.sorting ? 2 * (align_up(16 * L.sort_recs, 256) + align_up(L.sort_recs + 64, 256)) : 0;

    L.shape = shape;
    L.tpw = tpw;
    L.seg_cost = tu.seg_cost;
    L.virt = L.n_records + L.seg_cost * L.n_segs;
    L.tile = sweep_tile(shape);
    L.warps = kSweepShapes[shape].warps;
    const int cps = sweep_ctas_per_sm(shape, static_cast<int>(L.rmax));
    if (cps <= 0) return fail(TALP_GPU_ECUDA, "sweep kernel cannot be resident");
    const uint64_t tiles = (L.virt + L.tile - 1) / L.tile;
    uint64_t want = (tiles + tpw - 1) / tpw;
    const uint64_t max_warps = static_cast<uint64_t>(c->num_sms) * cps * L.warps;
    want = std::min(std::max<uint64_t>(want, 1), max_warps);
    L.grid = static_cast<int>((want + L.warps - 1) / L.warps);
    L.full_grid = static_cast<int>(max_warps / L.warps);
    L.spw = tu.spw;
    L.n_wrec = static_cast<uint32_t>(L.grid) * L.warps * static_cast<uint32_t>(L.spw > 0 ? L.spw : 1);
    L.n_wrec_cap = std::max<uint32_t>(L.n_wrec, L.sorting ? static_cast<uint32_t>(L.full_grid) * L.warps : 0u);

    for (size_t k = 0; k < nb; ++k)
        L.payload_words += 2ull * batches[k].n_ranks * batches[k].n_regions + L.mm[k] + sizeof(TraceDev) / 8;
    L.n_jobs_max = 8 * nb + 3;   // <= 8 per trace + seg flags + status + run log
    L.off_segs = 0;
    L.off_start = align_up(L.off_segs + sizeof(SegDesc) * L.n_segs, 256);
    L.off_send = align_up(L.off_start + sizeof(uint64_t) * (L.n_segs + 1), 256);
    L.off_jobs = align_up(L.off_send + sizeof(uint64_t) * (L.n_segs + 1), 256);
    L.off_rest = align_up(L.off_jobs + sizeof(FillJob) * L.n_jobs_max, 256);
    L.off_known = align_up(L.off_rest + sizeof(int64_t*) * (L.sorting ? L.n_segs : 0), 256);
    L.off_sctl = align_up(L.off_known + sizeof(uint64_t*) * (L.sorting ? L.n_segs : 0), 256);
    L.off_fin = align_up(L.off_sctl + sizeof(SortCtl), 256);
    L.off_pay = align_up(L.off_fin + sizeof(FinalizeJob) * L.n_fin, 256);
    L.up_bytes = align_up(L.off_pay + 8 * L.payload_words, 256);
    L.off_wrec = L.up_bytes;
    L.off_flags = align_up(L.off_wrec + sizeof(WarpRec) * L.n_wrec_cap, 256);
    L.off_gst = align_up(L.off_flags + sizeof(uint32_t) * (L.n_segs + 2), 256);
    L.off_bk = align_up(L.off_gst + 256, 256);
    L.off_slist = align_up(L.off_bk + 8 * L.n_backup_words, 256);
    L.off_srb = align_up(L.off_slist + 4 * L.sort_slots, 256);
    L.off_stb = align_up(L.off_srb + 8 * L.sort_slots, 256);
    L.off_smn = align_up(L.off_stb + 8 * (L.sort_slots + 1), 256);
    L.off_smx = align_up(L.off_smn + 8 * L.sort_slots, 256);
    L.off_hist = align_up(L.off_smx + 8 * L.sort_slots, 256);
    L.off_offs = align_up(L.off_hist + 4 * 256 * L.sort_tiles, 256);
    L.off_nruns = align_up(L.off_offs + 8 * 256 * L.sort_tiles, 256);
    L.off_runs = align_up(L.off_nruns + 4 * L.sort_slots, 256);
    L.off_fused = align_up(L.off_runs + 8 * (kMaxRuns + 1) * L.sort_slots, 256);
    L.off_given = align_up(L.off_fused + 4 * L.sort_slots, 256);
    L.off_fS = align_up(L.off_given + 4 * L.sort_slots, 256);
    L.off_fsb = align_up(L.off_fS + 4 * L.sort_slots, 256);
    L.off_fcb = align_up(L.off_fsb + 8 * (L.sort_slots + 1), 256);
    L.off_fpb = align_up(L.off_fcb + 8 * (L.sort_slots + 1), 256);
    L.off_fscb = align_up(L.off_fpb + 8 * L.sort_slots, 256);
    L.off_fsamp = align_up(L.off_fscb + 8 * (L.sort_slots + 1), 256);
    L.off_fsplit = align_up(L.off_fsamp + 8 * L.fms_samples, 256);
    L.off_fseg = align_up(L.off_fsplit + 8 * kMaxRuns * (L.fms_chunks + L.sort_slots), 256);
    L.off_fchunk = align_up(L.off_fseg + 4 * L.fms_chunks, 256);
    L.off_fscagg = align_up(L.off_fchunk + sizeof(FmsChunk) * L.fms_chunks, 256);
    L.off_ffix = align_up(L.off_fscagg + 16 * L.fms_super, 256);
    L.off_seen_n = align_up(L.off_ffix + sizeof(FmsFix) * L.fms_chunks, 256);
    L.off_seen_pos = align_up(L.off_seen_n + 4 * (L.sorting ? L.n_segs + 2 : 0), 256);
    L.off_rsegs = align_up(L.off_seen_pos + 8 * kMaxRuns * (L.sorting ? L.n_segs : 0), 256);
    L.off_rstart = align_up(L.off_rsegs + sizeof(SegDesc) * (L.sorting ? L.n_dev_segs : 0), 256);
    L.off_rrend = align_up(L.off_rstart + 8 * (L.sorting ? L.n_dev_segs + 1 : 0), 256);
    L.off_grp = align_up(L.off_rrend + 8 * (L.sorting ? L.n_dev_segs + 1 : 0), 256);
    L.off_mout = align_up(L.off_grp + 8 * kRunsStride * L.n_grouped, 256);
    L.ws_bytes = align_up(L.off_mout + sizeof(MetricsOut) * L.n_fin, 256);
    return TALP_GPU_OK;
}

// Find, reuse or create the trace states of an ingest.
talp_gpu_status get_traces(talp_gpu_ctx* c, const talp_gpu_trace_batch* batches, size_t nb, cudaStream_t stream,
                           std::vector<TraceState*>& ts) {
    ts.assign(nb, nullptr);
    for (size_t k = 0; k < nb; ++k) {
        const talp_gpu_trace_batch& b = batches[k];
        // a new trace of this id ends the old one's held-back raw records
        if (!(b.flags & TALP_GPU_APPEND) && !c->raw_inner) raw_hold_drop(c, b.trace_id);
        auto it = c->traces.find(b.trace_id);
        if (it != c->traces.end() && same_shape(it->second, b)) {
            ts[k] = it->second;
            continue;
        }
        if (it != c->traces.end()) {
            cudaStreamSynchronize(stream);
            free_trace(c, it->second);
            c->traces.erase(it);
        }
        TraceState* t = nullptr;
        TALP_TRY(alloc_trace(c, b.trace_id, b.n_ranks, b.devices_per_rank, b.n_regions, &t));
        c->traces[b.trace_id] = t;
        ts[k] = t;
    }
    return TALP_GPU_OK;
}

const uint8_t* floor16(const uint8_t* p) {
    return reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(p) & ~static_cast<uintptr_t>(15));
}

// Write the upload part of the workspace (segment table, starts, jobs,
// payload, sort control, finalize jobs) into `up`, with device addresses in
// the workspace `wsd`.  Host-pointer records are copied into `stg` on
// `stream`.  `mout_user`: where finalize writes (null: the workspace).
talp_gpu_status fill_ingest(talp_gpu_ctx* c, const talp_gpu_trace_batch* batches, size_t nb, Layout& L,
                            const std::vector<TraceState*>& ts, char* up, char* wsd, char* stg, char* sortbuf,
                            cudaStream_t stream) {
    std::vector<const int64_t*> hse(nb), dse(nb);
    std::vector<const uint8_t*> hst(nb), dtg(nb), hst_end(nb), dtg_end(nb);
    size_t so = 0;
    for (size_t k = 0; k < nb; ++k) {
        const talp_gpu_trace_batch& b = batches[k];
        if (b.flags & TALP_GPU_DEVICE_PTRS) {
            hse[k] = b.host_se;
            dse[k] = b.dev_se;
            hst[k] = b.host_state;
            dtg[k] = b.dev_tag;
        } else {
            auto put = [&](const void* src, size_t bytes) -> char* {
                char* d = stg + so;
                if (bytes) {
                    cudaError_t e = cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, stream);
                    if (e != cudaSuccess) return nullptr;
                }
                so = align_up(so + bytes, 16);
                return d;
            };
            char* a = put(b.host_se, L.nh[k] * 16);
            char* bb = put(b.dev_se, L.nd[k] * 16);
            char* cc = put(b.host_state, L.nh[k]);
            char* dd = put(b.dev_tag, L.nd[k]);
            if (!a || !bb || !cc || !dd) return cuda_fail(cudaGetLastError(), "cudaMemcpyAsync (records)");
            hse[k] = reinterpret_cast<const int64_t*>(a);
            dse[k] = reinterpret_cast<const int64_t*>(bb);
            hst[k] = reinterpret_cast<const uint8_t*>(cc);
            dtg[k] = reinterpret_cast<const uint8_t*>(dd);
        }
        hst_end[k] = floor16(hst[k] + L.nh[k]);
        dtg_end[k] = floor16(dtg[k] + L.nd[k]);
    }

    SegDesc* sd = reinterpret_cast<SegDesc*>(up + L.off_segs);
    uint64_t* sstart = reinterpret_cast<uint64_t*>(up + L.off_start);
    uint64_t* send = reinterpret_cast<uint64_t*>(up + L.off_send);
    FillJob* jobs = reinterpret_cast<FillJob*>(up + L.off_jobs);
    const int64_t** restore = reinterpret_cast<const int64_t**>(up + L.off_rest);
    const uint64_t** known = reinterpret_cast<const uint64_t**>(up + L.off_known);
    FinalizeJob* fin = reinterpret_cast<FinalizeJob*>(up + L.off_fin);
    int64_t* pay = reinterpret_cast<int64_t*>(up + L.off_pay);
    int64_t* pay_dev = reinterpret_cast<int64_t*>(wsd + L.off_pay);
    uint32_t* seg_flags = reinterpret_cast<uint32_t*>(wsd + L.off_flags);
    uint32_t* gstatus = reinterpret_cast<uint32_t*>(wsd + L.off_gst);
    MetricsOut* mout = reinterpret_cast<MetricsOut*>(wsd + L.off_mout);
    size_t pw = 0, bk_used = 0, nf = 0;
    uint32_t nj = 0;
    uint64_t si = 0, pos = 0, gi = 0;   // gi: grouped device segments so far
    size_t presort_at = 0;   // first device of this batch in c->raw_presort
    for (size_t k = 0; k < nb; ++k) {
        const talp_gpu_trace_batch& b = batches[k];
        TraceState* t = ts[k];
        const bool append = (b.flags & TALP_GPU_APPEND) != 0;
        const uint32_t n = t->n, m = t->m, R = t->R;
        int64_t* cin = t->carry[t->cur];
        int64_t* cout = t->carry[t->cur ^ 1];
        int64_t* bkd = nullptr;   // pre-ingest device sums (APPEND + sorting)
        // windows: transpose [R][n][2] -> [n][R][2]
        int64_t* hw = pay + pw;
        for (uint32_t i = 0; i < n; ++i)
            for (uint32_t r = 0; r < R; ++r) {
                hw[(i * R + r) * 2 + 0] = b.region_window[(static_cast<size_t>(r) * n + i) * 2 + 0];
                hw[(i * R + r) * 2 + 1] = b.region_window[(static_cast<size_t>(r) * n + i) * 2 + 1];
            }
        jobs[nj++] = FillJob{t->hwin, 2ull * n * R, 0, pay_dev + pw};
        pw += 2ull * n * R;
        int64_t* dr = pay + pw;
        {
            uint64_t g = 0;
            for (uint32_t i = 0; i < n; ++i)
                for (uint32_t q = 0; q < b.devices_per_rank[i]; ++q) dr[g++] = i;
        }
        if (m) jobs[nj++] = FillJob{t->dev_rank, m, 0, pay_dev + pw};
        pw += m;
        TraceDev td{};
        td.trace_id = t->id;
        td.n = n;
        td.m = m;
        td.R = R;
        td.hsum = t->hsum;
        td.dsum = t->dsum;
        td.hwin = t->hwin;
        td.dev_rank = t->dev_rank;
        td.status = t->status;
        memcpy(pay + pw, &td, sizeof(TraceDev));
        jobs[nj++] = FillJob{reinterpret_cast<int64_t*>(t->tdev), sizeof(TraceDev) / 8, 0, pay_dev + pw};
        pw += sizeof(TraceDev) / 8;
        if (!append) {
            jobs[nj++] = FillJob{t->hsum, 3ull * n * R, 0, nullptr};
            if (m) jobs[nj++] = FillJob{t->dsum, 3ull * m * R, 0, nullptr};
            if (m) jobs[nj++] = FillJob{cin, 3ull * m, NEG_INF, nullptr};
            if (m) jobs[nj++] = FillJob{cout, 3ull * m, NEG_INF, nullptr};
            jobs[nj++] = FillJob{reinterpret_cast<int64_t*>(t->status), 1, 0, nullptr};
        } else {
            if (m) jobs[nj++] = FillJob{cout, 3ull * m, 0, cin};
            if (!(b.flags & TALP_GPU_SORTED_BY_START) && m) {
                // a device segment that gets sorted is re-swept from its sums
                // before this slice: keep a copy of them
                bkd = reinterpret_cast<int64_t*>(wsd + L.off_bk) + bk_used;
                bk_used += 3ull * R * m;
                jobs[nj++] = FillJob{bkd, 3ull * m * R, 0, t->dsum};
            }
        }
        for (uint32_t r = 0; r < R && L.n_fin; ++r) {
            fin[nf] = FinalizeJob{t->tdev, mout + nf, r, 0};
            ++nf;
        }
        const uint8_t sflag = (b.flags & TALP_GPU_SORTED_BY_START) ? 0 : kSegSortable;
        // device segments, then host segments
        for (uint32_t g = 0; g < m; ++g) {
            SegDesc& s = sd[si];
            memset(&s, 0, sizeof(SegDesc));
            const uint64_t o = b.dev_off[g];
            s.se = dse[k] + 2 * o;
            s.tag = dtg[k] + o;
            s.tag_limit = dtg_end[k];
            s.sums = t->dsum + static_cast<size_t>(g) * R * 3;
            s.win = t->hwin + static_cast<size_t>(dr[g]) * R * 2;
            s.status = t->status;
            s.carry_in = cin + 3ull * g;
            s.carry_out = cout + 3ull * g;
            s.n = b.dev_off[g + 1] - o;
            s.R = static_cast<uint16_t>(R);
            s.is_host = 0;
            s.pad[0] = sflag;
            if (L.sorting) restore[si] = bkd ? bkd + static_cast<size_t>(g) * R * 3 : nullptr;
            sstart[si] = pos;
            const bool grouped = sflag && (b.flags & TALP_GPU_GROUPED_BY_STREAM);
            const bool presort = (b.flags & TALP_GPU_NOT_SORTED) || grouped ||
                                 (c->raw_inner && presort_at + g < c->raw_presort.size() && c->raw_presort[presort_at + g]);
            if (L.sorting) {
                // a raw lane's runs are its streams, known from the adapter; a
                // grouped device's runs are its stream groups, found on the GPU
                // from its tags before the sort stage
                known[si] = (sflag && presort && c->raw_inner && c->raw_runs)
                                ? c->raw_runs + static_cast<size_t>(presort_at + g) * kRunsStride
                                : nullptr;
                if (grouped) {
                    known[si] = reinterpret_cast<const uint64_t*>(wsd + L.off_grp) + gi * kRunsStride;
                    s.pad[0] |= kSegGrouped;
                    ++gi;
                }
            }
            if (sflag && presort) {
                s.pad[0] |= kSegPresort;   // not in the first sweep: sorted, then swept
                send[si] = pos;
            } else {
                send[si] = pos + s.n;
                pos += s.n + L.seg_cost;
            }
            ++si;
        }
        presort_at += m;
        for (uint32_t i = 0; i < n; ++i) {
            SegDesc& s = sd[si];
            memset(&s, 0, sizeof(SegDesc));
            const uint64_t o = b.host_off[i];
            s.se = hse[k] + 2 * o;
            s.tag = hst[k] + o;
            s.tag_limit = hst_end[k];
            s.sums = t->hsum + static_cast<size_t>(i) * R * 3;
            s.win = t->hwin + static_cast<size_t>(i) * R * 2;
            s.status = t->status;
            s.n = b.host_off[i + 1] - o;
            s.R = static_cast<uint16_t>(R);
            s.is_host = 1;
            if (L.sorting) {
                restore[si] = nullptr;
                known[si] = nullptr;
            }
            sstart[si] = pos;
            send[si] = pos + s.n;
            pos += s.n + L.seg_cost;
            ++si;
        }
    }
    sstart[si] = pos;
    send[si] = pos;
    jobs[nj++] = FillJob{reinterpret_cast<int64_t*>(seg_flags), (L.n_segs + 2) / 2, 0, nullptr};
    jobs[nj++] = FillJob{reinterpret_cast<int64_t*>(gstatus), 2, 0, nullptr};   // status, pad, slice ticket
    if (L.sorting) jobs[nj++] = FillJob{reinterpret_cast<int64_t*>(wsd + L.off_seen_n), (L.n_segs + 2) / 2, 0, nullptr};
    if (nj > L.n_jobs_max || pw > L.payload_words || si != L.n_segs || bk_used > L.n_backup_words || nf != L.n_fin ||
        gi != L.n_grouped)
        return fail(TALP_GPU_ECUDA, "internal: upload table overflow");
    L.nj = nj;
    if (L.sorting) {
        SortCtl sc{};
        sc.list = reinterpret_cast<uint32_t*>(wsd + L.off_slist);
        sc.rec_base = reinterpret_cast<uint64_t*>(wsd + L.off_srb);
        sc.tile_base = reinterpret_cast<uint64_t*>(wsd + L.off_stb);
        sc.mn = reinterpret_cast<int64_t*>(wsd + L.off_smn);
        sc.mx = reinterpret_cast<int64_t*>(wsd + L.off_smx);
        sc.hist = reinterpret_cast<uint32_t*>(wsd + L.off_hist);
        sc.offs = reinterpret_cast<uint64_t*>(wsd + L.off_offs);
        sc.nruns = reinterpret_cast<uint32_t*>(wsd + L.off_nruns);
        sc.runs = reinterpret_cast<uint64_t*>(wsd + L.off_runs);
        sc.fused = reinterpret_cast<uint32_t*>(wsd + L.off_fused);
        sc.given = reinterpret_cast<uint32_t*>(wsd + L.off_given);
        sc.known = reinterpret_cast<const uint64_t* const*>(wsd + L.off_known);
        sc.seen_n = reinterpret_cast<const uint32_t*>(wsd + L.off_seen_n);
        sc.seen_pos = reinterpret_cast<const uint64_t*>(wsd + L.off_seen_pos);
        sc.fms_S = reinterpret_cast<uint32_t*>(wsd + L.off_fS);
        sc.fms_samp_base = reinterpret_cast<uint64_t*>(wsd + L.off_fsb);
        sc.fms_chunk_base = reinterpret_cast<uint64_t*>(wsd + L.off_fcb);
        sc.fms_split_base = reinterpret_cast<uint64_t*>(wsd + L.off_fpb);
        sc.fms_sc_base = reinterpret_cast<uint64_t*>(wsd + L.off_fscb);
        sc.fms_samp = reinterpret_cast<int64_t*>(wsd + L.off_fsamp);
        sc.fms_split = reinterpret_cast<uint64_t*>(wsd + L.off_fsplit);
        sc.fms_chunk_seg = reinterpret_cast<uint32_t*>(wsd + L.off_fseg);
        sc.fms_chunk = reinterpret_cast<FmsChunk*>(wsd + L.off_fchunk);
        sc.fms_sc_agg = reinterpret_cast<int64_t*>(wsd + L.off_fscagg);
        sc.fms_fix = reinterpret_cast<FmsFix*>(wsd + L.off_ffix);
        const size_t se_b = align_up(16 * L.sort_recs, 256), tg_b = align_up(L.sort_recs + 64, 256);
        for (int q = 0; q < 2; ++q) {
            char* base = sortbuf + q * (se_b + tg_b);
            sc.buf_se[q] = reinterpret_cast<int64_t*>(base);
            sc.buf_tag[q] = reinterpret_cast<uint8_t*>(base + se_b);
            sc.buf_tag_limit[q] = floor16(reinterpret_cast<const uint8_t*>(base + se_b + tg_b));
        }
        sc.restore = reinterpret_cast<const int64_t* const*>(wsd + L.off_rest);
        memcpy(up + L.off_sctl, &sc, sizeof(SortCtl));
    }
    (void)c;
    return TALP_GPU_OK;
}

// Upload and the launch sequence of an ingest (capturable).
talp_gpu_status enqueue_ingest(talp_gpu_ctx* c, const Layout& L, const char* up, char* wsd, cudaStream_t stream,
                               bool profile, uint64_t* launches, bool upload = true) {
    uint64_t nl = 0;
    if (upload) TALP_CUDA(cudaMemcpyAsync(wsd, up, L.up_bytes, cudaMemcpyHostToDevice, stream));
    TALP_CUDA(launch_prep(reinterpret_cast<const FillJob*>(wsd + L.off_jobs), L.nj, stream));
    ++nl;
    const SegDesc* dsegs = reinterpret_cast<const SegDesc*>(wsd + L.off_segs);
    const uint64_t* dstart = reinterpret_cast<const uint64_t*>(wsd + L.off_start);
    const uint64_t* dsend = reinterpret_cast<const uint64_t*>(wsd + L.off_send);
    WarpRec* wrec = reinterpret_cast<WarpRec*>(wsd + L.off_wrec);
    uint32_t* seg_flags = reinterpret_cast<uint32_t*>(wsd + L.off_flags);
    uint32_t* gstatus = reinterpret_cast<uint32_t*>(wsd + L.off_gst);
    if (L.n_records > 0) {
        if (L.n_grouped) {   // the runs of grouped devices, from their tags
            TALP_CUDA(launch_group_runs(dsegs, static_cast<uint32_t>(L.n_segs),
                                        reinterpret_cast<const uint64_t* const*>(wsd + L.off_known), stream));
            ++nl;
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (profile) {
            e0 = take_event(c);
            e1 = take_event(c);
            TALP_CUDA(cudaEventRecord(e0, stream));
        }
        // with a sort stage to follow, segments found out of order are not
        // computed any further, only scanned for where their order descends
        const RunLog rl = L.sorting ? RunLog{reinterpret_cast<uint32_t*>(wsd + L.off_seen_n),
                                             reinterpret_cast<uint64_t*>(wsd + L.off_seen_pos)}
                                    : RunLog{nullptr, nullptr};
        TALP_CUDA(launch_sweep(L.shape, static_cast<int>(L.rmax), L.grid, dsegs, dstart, dsend,
                               static_cast<uint32_t>(L.n_segs), wrec, seg_flags, gstatus, c->wait_limit, L.sorting,
                               rl, L.spw > 0 ? L.n_wrec : 0u, L.spw > 0 ? gstatus + 2 : nullptr, stream));
        if (profile) {
            TALP_CUDA(cudaEventRecord(e1, stream));
            c->ev_pending.emplace_back(e0, e1);
            c->ev_records.push_back(L.n_records);
        }
        TALP_CUDA(launch_fixup(dsegs, dstart, wrec, L.n_wrec, seg_flags, L.sorting, rl, stream));
        nl += 2;
        if (L.sorting) {
            // a2: sort the device segments found out of order, re-sweep them
            SortCtl* sctl = reinterpret_cast<SortCtl*>(wsd + L.off_sctl);
            SegDesc* rsegs = reinterpret_cast<SegDesc*>(wsd + L.off_rsegs);
            uint64_t* rstart = reinterpret_cast<uint64_t*>(wsd + L.off_rstart);
            uint64_t* rrend = reinterpret_cast<uint64_t*>(wsd + L.off_rrend);
            const uint64_t gt = std::min<uint64_t>(L.sort_tiles, static_cast<uint64_t>(c->num_sms) * 8);
            const uint64_t gs = std::min<uint64_t>(L.sort_slots, static_cast<uint64_t>(c->num_sms) * 4);
            cudaEvent_t s0 = nullptr, s1 = nullptr;
            if (profile) {
                s0 = take_event(c);
                s1 = take_event(c);
                TALP_CUDA(cudaEventRecord(s0, stream));
            }
            TALP_CUDA(launch_sort_stage(dsegs, static_cast<uint32_t>(L.n_segs), static_cast<uint32_t>(L.n_dev_segs),
                                        seg_flags, sctl, rsegs, rstart, rrend,
                                        static_cast<int>(std::max<uint64_t>(gt, 1)),
                                        static_cast<int>(std::max<uint64_t>(gs, 1)), gstatus, c->wait_limit, stream));
            if (profile) {
                TALP_CUDA(cudaEventRecord(s1, stream));
                c->sort_ev_pending.emplace_back(s0, s1);
            }
            TALP_CUDA(launch_sweep(L.shape, static_cast<int>(L.rmax), L.full_grid, rsegs, rstart, rrend,
                                   static_cast<uint32_t>(L.n_dev_segs), wrec, seg_flags, gstatus, c->wait_limit,
                                   false, RunLog{nullptr, nullptr}, 0u, nullptr, stream));
            TALP_CUDA(launch_fixup(rsegs, rstart, wrec, static_cast<uint32_t>(L.full_grid) * L.warps, seg_flags,
                                   false, RunLog{nullptr, nullptr}, stream));
            nl += 2 + 1 + 4 + 24 + 1 + 2;
        }
    }
    if (L.n_fin) {
        TALP_CUDA(launch_finalize(reinterpret_cast<const FinalizeJob*>(wsd + L.off_fin),
                                  static_cast<uint32_t>(L.n_fin), stream));
        ++nl;
    }
    if (launches) *launches = nl;
    return TALP_GPU_OK;
}

talp_gpu_status check_metrics_flags(const talp_gpu_metrics* out, size_t n) {
    for (size_t k = 0; k < n; ++k) {
        const uint32_t f = out[k].flags;
        if (f & TALP_GPU_M_TIMEOUT) return fail(TALP_GPU_ETIMEDOUT, "a device-side wait ran out during ingest");
        if (f & (TALP_GPU_M_INVALID | TALP_GPU_M_UNSORTED))
            return fail(TALP_GPU_EINVAL, (f & TALP_GPU_M_INVALID) ? "invalid record (end < start or bad kind/state)"
                                                                 : "device records out of start order");
    }
    return TALP_GPU_OK;
}

// Default segment cost in records: a segment switch costs about two tiles
// of streaming, and every window boundary (2 per region beyond the first)
// that falls inside the segment's time range costs one clipped re-pass of
// the tile holding it.  Short segments are mostly such tiles; without this
// term the slices of warps full of short segments run several times longer
// than the others.
uint64_t default_seg_cost(uint32_t rmax, uint32_t tile) {
    return 512 + 64ull * rmax + 2ull * (rmax - 1) * tile;
}

Tuning pick_tuning(talp_gpu_ctx* c, const talp_gpu_trace_batch* batches, size_t nb) {
    Tuning tu = c->defaults;
    uint32_t rmax = 1;
    for (size_t k = 0; k < nb; ++k) rmax = std::max(rmax, batches[k].n_regions);
    if (!tu.seg_cost) tu.seg_cost = default_seg_cost(rmax, static_cast<uint32_t>(sweep_tile(tu.shape)));
    if (c->shape_forced || c->tune.empty()) return tu;
    uint64_t recs = 0, segs = 0;
    bool sorting = false;
    for (size_t k = 0; k < nb; ++k) {
        const talp_gpu_trace_batch& b = batches[k];
        uint64_t m = 0;
        for (uint32_t i = 0; i < b.n_ranks; ++i) m += b.devices_per_rank[i];
        recs += b.host_off[b.n_ranks] + b.dev_off[m];
        segs += m + b.n_ranks;
        sorting |= !(b.flags & TALP_GPU_SORTED_BY_START);
    }
    auto it = c->tune.find(size_class(recs, segs, sorting));
    if (it != c->tune.end()) tu = it->second;
    return tu;
}

}  // namespace

// ===================================================================== ABI

extern "C" {

const char* talp_gpu_last_error(void) { return g_last_error.c_str(); }

talp_gpu_status talp_gpu_create(talp_gpu_ctx** out, int device, size_t hbm_budget_bytes) {
    if (!out) return fail(TALP_GPU_EINVAL, "null out");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(TALP_GPU_EINVAL, "bad device index");
    TALP_CUDA(cudaSetDevice(device));
    talp_gpu_ctx* c = new talp_gpu_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->budget = hbm_budget_bytes ? hbm_budget_bytes : static_cast<size_t>(fr * 0.9);
    cudaEventCreateWithFlags(&c->ev_up, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&c->ev_upf, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&c->ev_ws, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&c->ev_raw, cudaEventDisableTiming);
    cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    // overrides of the sweep tuning (benchmarks and tests)
    // device-side wait limit in clock cycles; a negative value makes every
    // sweep report a time-out at its first wait (tests of the failure path)
    if (const char* s = getenv("TALP_GPU_WAIT_LIMIT")) c->wait_limit = strtoll(s, nullptr, 10);
    if (const char* s = getenv("TALP_GPU_SWEEP_SHAPE")) {
        c->defaults.shape = atoi(s) % kNumSweepShapes;
        c->shape_forced = true;
    }
    if (const char* s = getenv("TALP_GPU_TILES_PER_WARP")) {
        c->defaults.tpw = atoi(s) > 0 ? atoi(s) : 4;
        c->shape_forced = true;
    }
    if (const char* s = getenv("TALP_GPU_SEG_COST")) {
        c->defaults.seg_cost = strtoull(s, nullptr, 10);
        c->shape_forced = true;
    }
    if (const char* s = getenv("TALP_GPU_SLICES_PER_WARP")) {
        c->defaults.spw = atoi(s) > 0 ? atoi(s) : 0;
        c->shape_forced = true;
    }
    *out = c;
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_destroy(talp_gpu_ctx* c) {
    if (!c) return TALP_GPU_OK;
    if (c->dependents > 0) return fail(TALP_GPU_EBUSY, "plans or servers still use this context");
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    raw_hold_drop(c, TALP_GPU_ALL);
    for (auto& kv : c->traces) free_trace(c, kv.second);
    c->traces.clear();
    dev_free(c, c->ws.p, c->ws.cap);
    dev_free(c, c->stage.p, c->stage.cap);
    dev_free(c, c->sortbuf.p, c->sortbuf.cap);
    dev_free(c, c->raw.p, c->raw.cap);
    if (c->up.p) cudaFreeHost(c->up.p);
    if (c->upf.p) cudaFreeHost(c->upf.p);
    if (c->down.p) cudaFreeHost(c->down.p);
    if (c->ev_up) cudaEventDestroy(c->ev_up);
    if (c->ev_upf) cudaEventDestroy(c->ev_upf);
    if (c->ev_ws) cudaEventDestroy(c->ev_ws);
    if (c->ev_raw) cudaEventDestroy(c->ev_raw);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (auto& pr : c->ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto& pr : c->sort_ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_ingest_events(talp_gpu_ctx* c, const talp_gpu_trace_batch* batches, size_t nb,
                                       void* stream_) {
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    if (nb == 0) return TALP_GPU_OK;
    if (!batches) return fail(TALP_GPU_EINVAL, "null batches");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    TALP_CUDA(cudaSetDevice(c->device));

    Layout L;
    TALP_TRY(size_ingest(c, batches, nb, pick_tuning(c, batches, nb), false, L));

    // admission: everything this ingest would add, before any allocation
    size_t extra = L.new_bytes;
    if (c->ws.cap < L.ws_bytes) extra += grow_size(L.ws_bytes) - c->ws.cap;
    if (c->stage.cap < L.stage_bytes) extra += grow_size(L.stage_bytes) - c->stage.cap;
    if (c->sortbuf.cap < L.sortbuf_bytes) extra += grow_size(L.sortbuf_bytes) - c->sortbuf.cap;
    if (c->held + extra > c->budget)
        return fail(TALP_GPU_ENOMEM, "admission: the ingest needs " + std::to_string(extra) +
                                         " more device bytes than the budget leaves");

    // the previous ingest must be done with the workspace/staging before reuse
    if (c->ws_used) TALP_CUDA(cudaStreamWaitEvent(stream, c->ev_ws, 0));
    TALP_TRY(grow(c, c->ws, L.ws_bytes));
    if (L.stage_bytes) TALP_TRY(grow(c, c->stage, L.stage_bytes));
    if (L.sortbuf_bytes) TALP_TRY(grow(c, c->sortbuf, L.sortbuf_bytes));
    TALP_CUDA(cudaEventSynchronize(c->ev_up));   // upload scratch no longer read by a pending copy
    TALP_TRY(grow_pinned(c->up, L.up_bytes));

    std::vector<TraceState*> ts;
    TALP_TRY(get_traces(c, batches, nb, stream, ts));
    char* up = static_cast<char*>(c->up.p);
    char* wsd = static_cast<char*>(c->ws.p);
    TALP_TRY(fill_ingest(c, batches, nb, L, ts, up, wsd, static_cast<char*>(c->stage.p),
                         static_cast<char*>(c->sortbuf.p), stream));
    uint64_t nl = 0;
    TALP_TRY(enqueue_ingest(c, L, up, wsd, stream, c->profiling, &nl));
    c->kernel_launches += nl;
    TALP_CUDA(cudaEventRecord(c->ev_up, stream));
    TALP_CUDA(cudaEventRecord(c->ev_ws, stream));
    c->ws_used = true;
    for (size_t k = 0; k < nb; ++k) ts[k]->cur ^= 1;
    return TALP_GPU_OK;
}

static talp_gpu_status finalize_common(talp_gpu_ctx* c, const uint64_t* ids, size_t n, uint32_t region,
                                       MetricsOut* out_dev_user, talp_gpu_metrics* out_host, cudaStream_t stream,
                                       bool sync) {
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    if (n == 0) return TALP_GPU_OK;
    TALP_CUDA(cudaSetDevice(c->device));
    std::vector<FinalizeJob> jobs;
    for (size_t k = 0; k < n; ++k) {
        auto it = c->traces.find(ids[k]);
        if (it == c->traces.end()) return fail(TALP_GPU_ENOTFOUND, "unknown trace id " + std::to_string(ids[k]));
        TraceState* t = it->second;
        if (region == TALP_GPU_ALL_REGIONS) {
            if (n != 1) return fail(TALP_GPU_EINVAL, "TALP_GPU_ALL_REGIONS takes one trace");
            for (uint32_t r = 0; r < t->R; ++r) jobs.push_back(FinalizeJob{t->tdev, nullptr, r, 0});
        } else {
            if (region >= t->R) return fail(TALP_GPU_EINVAL, "region out of range");
            jobs.push_back(FinalizeJob{t->tdev, nullptr, region, 0});
        }
    }
    const size_t nj = jobs.size();
    const size_t jb = align_up(sizeof(FinalizeJob) * nj, 256);
    if (c->ws_used) TALP_CUDA(cudaStreamWaitEvent(stream, c->ev_ws, 0));
    TALP_TRY(grow(c, c->ws, jb + sizeof(MetricsOut) * nj));
    MetricsOut* res = reinterpret_cast<MetricsOut*>(static_cast<char*>(c->ws.p) + jb);
    for (size_t k = 0; k < nj; ++k) jobs[k].out = out_dev_user ? out_dev_user + k : res + k;
    TALP_CUDA(cudaEventSynchronize(c->ev_upf));
    TALP_TRY(grow_pinned(c->upf, jb));
    memcpy(c->upf.p, jobs.data(), sizeof(FinalizeJob) * nj);
    TALP_CUDA(cudaMemcpyAsync(c->ws.p, c->upf.p, sizeof(FinalizeJob) * nj, cudaMemcpyHostToDevice, stream));
    TALP_CUDA(cudaEventRecord(c->ev_upf, stream));
    TALP_CUDA(launch_finalize(static_cast<const FinalizeJob*>(c->ws.p), static_cast<uint32_t>(nj), stream));
    ++c->kernel_launches;
    if (!sync) {
        TALP_CUDA(cudaEventRecord(c->ev_ws, stream));
        c->ws_used = true;
        return TALP_GPU_OK;
    }
    TALP_TRY(grow_pinned(c->down, sizeof(MetricsOut) * nj));
    TALP_CUDA(cudaMemcpyAsync(c->down.p, res, sizeof(MetricsOut) * nj, cudaMemcpyDeviceToHost, stream));
    TALP_CUDA(cudaEventRecord(c->ev_ws, stream));
    c->ws_used = true;
    TALP_CUDA(cudaStreamSynchronize(stream));
    memcpy(out_host, c->down.p, sizeof(MetricsOut) * nj);
    return check_metrics_flags(out_host, nj);
}

talp_gpu_status talp_gpu_region_metrics(talp_gpu_ctx* c, uint64_t trace_id, uint32_t region,
                                        talp_gpu_metrics* out_host, void* stream) {
    if (!out_host) return fail(TALP_GPU_EINVAL, "null out");
    return finalize_common(c, &trace_id, 1, region, nullptr, out_host, static_cast<cudaStream_t>(stream), true);
}

talp_gpu_status talp_gpu_region_metrics_batch(talp_gpu_ctx* c, const uint64_t* ids, size_t n, uint32_t region,
                                              talp_gpu_metrics* out_host, void* stream) {
    if (!out_host || (n && !ids)) return fail(TALP_GPU_EINVAL, "null argument");
    if (region == TALP_GPU_ALL_REGIONS && n != 1) return fail(TALP_GPU_EINVAL, "ALL_REGIONS takes one trace");
    return finalize_common(c, ids, n, region, nullptr, out_host, static_cast<cudaStream_t>(stream), true);
}

talp_gpu_status talp_gpu_region_metrics_device(talp_gpu_ctx* c, const uint64_t* ids, size_t n, uint32_t region,
                                               talp_gpu_metrics* out_device, void* stream) {
    if (!out_device || (n && !ids)) return fail(TALP_GPU_EINVAL, "null argument");
    if ((reinterpret_cast<uintptr_t>(out_device) & 7u) != 0) return fail(TALP_GPU_EINVAL, "out_device misaligned");
    return finalize_common(c, ids, n, region, reinterpret_cast<MetricsOut*>(out_device), nullptr,
                           static_cast<cudaStream_t>(stream), false);
}

talp_gpu_status talp_gpu_metrics_combine(talp_gpu_ctx* c, const talp_gpu_metrics* parts, size_t n_parts,
                                         talp_gpu_metrics* out_host, void* stream_) {
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    if (!parts || !out_host || n_parts == 0) return fail(TALP_GPU_EINVAL, "null argument or no parts");
    if (n_parts > (1u << 20)) return fail(TALP_GPU_EINVAL, "more than 2^20 parts");
    for (size_t k = 1; k < n_parts; ++k)
        if (parts[k].trace_id != parts[0].trace_id || parts[k].region != parts[0].region)
            return fail(TALP_GPU_EINVAL, "parts of different traces or regions");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    TALP_CUDA(cudaSetDevice(c->device));
    const size_t pb = align_up(sizeof(MetricsOut) * n_parts, 256);
    if (c->ws_used) TALP_CUDA(cudaStreamWaitEvent(stream, c->ev_ws, 0));
    TALP_TRY(grow(c, c->ws, pb + sizeof(MetricsOut)));
    MetricsOut* dparts = static_cast<MetricsOut*>(c->ws.p);
    MetricsOut* dres = reinterpret_cast<MetricsOut*>(static_cast<char*>(c->ws.p) + pb);
    TALP_CUDA(cudaEventSynchronize(c->ev_up));
    TALP_TRY(grow_pinned(c->up, pb));
    memcpy(c->up.p, parts, sizeof(MetricsOut) * n_parts);
    TALP_CUDA(cudaMemcpyAsync(dparts, c->up.p, sizeof(MetricsOut) * n_parts, cudaMemcpyHostToDevice, stream));
    TALP_CUDA(cudaEventRecord(c->ev_up, stream));
    TALP_CUDA(launch_combine(dparts, static_cast<uint32_t>(n_parts), dres, stream));
    ++c->kernel_launches;
    TALP_TRY(grow_pinned(c->down, sizeof(MetricsOut)));
    TALP_CUDA(cudaMemcpyAsync(c->down.p, dres, sizeof(MetricsOut), cudaMemcpyDeviceToHost, stream));
    TALP_CUDA(cudaEventRecord(c->ev_ws, stream));
    c->ws_used = true;
    TALP_CUDA(cudaStreamSynchronize(stream));
    memcpy(out_host, c->down.p, sizeof(MetricsOut));
    return check_metrics_flags(out_host, 1);
}

}  // extern "C"

namespace {

// Held-back raw records of a trace: its shape, each stream's last delivered
// start and declared-stream masks, and the held records (ping-pong buffers;
// rank r's held records at buf[cur] + off[r], cnt[r] of them).
struct RawHold {
    uint32_t n = 0;
    std::vector<uint32_t> dpr;
    std::vector<uint32_t> smask;   // [n][kRawMaxDevices]
    DevBuf ls;                     // int64 [n][kRawBuckets]
    bool fresh = true;             // ls not written yet
    DevBuf buf[2];
    size_t o_tag[2] = {0, 0}, o_dev[2] = {0, 0};   // byte offsets of the tags and devices in buf[k]
    int cur = 0;
    std::vector<uint64_t> off, cnt;
};

// held-record buffer for up to cap records: rows, then tags, then devices
size_t hold_tag_at(uint64_t cap) { return align_up(16 * cap, 256); }
size_t hold_dev_at(uint64_t cap) { return align_up(hold_tag_at(cap) + cap, 256); }
size_t hold_bytes(uint64_t cap) { return align_up(hold_dev_at(cap) + cap, 256) + 256; }

}  // namespace

void talp::raw_hold_drop(talp_gpu_ctx* c, uint64_t trace_id) {
    auto& m = c->holds;
    auto drop = [&](RawHold* h) {
        dev_free(c, h->ls.p, h->ls.cap);
        dev_free(c, h->buf[0].p, h->buf[0].cap);
        dev_free(c, h->buf[1].p, h->buf[1].cap);
        delete h;
    };
    if (trace_id == TALP_GPU_ALL) {
        for (auto& kv : m) drop(kv.second);
        m.clear();
        return;
    }
    auto it = m.find(trace_id);
    if (it == m.end()) return;
    drop(it->second);
    m.erase(it);
}

uint64_t talp::raw_held_records(talp_gpu_ctx* c, uint64_t trace_id) {
    auto it = c->holds.find(trace_id);
    if (it == c->holds.end()) return 0;
    uint64_t t = 0;
    for (uint64_t v : it->second->cnt) t += v;
    return t;
}

extern "C" {

talp_gpu_status talp_gpu_raw_held(talp_gpu_ctx* c, uint64_t trace_id, uint64_t* out_host) {
    if (!c || !out_host) return fail(TALP_GPU_EINVAL, "null argument");
    *out_host = raw_held_records(c, trace_id);
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_ingest_raw(talp_gpu_ctx* c, const talp_gpu_raw_batch* rb, size_t nb, void* stream_) {
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    if (nb == 0) return TALP_GPU_OK;
    if (!rb) return fail(TALP_GPU_EINVAL, "null batches");
    const bool dev_ptrs = (rb[0].flags & TALP_GPU_DEVICE_PTRS) != 0;
    const uint64_t tile = static_cast<uint64_t>(raw_tile_records());
    auto& holds = c->holds;

    // pass 1: headers, sizes and the hold state each batch continues
    std::vector<RawHold*> hs(nb, nullptr);      // hold state read (held records prepended)
    std::vector<bool> hb(nb, false);            // batch holds back
    std::vector<uint64_t> out_base(nb), hbase(nb), m_of(nb);
    uint64_t nr = 0, outn = 0, nh = 0, mtot = 0, nt = 0, nrk = 0;
    bool any_hold = false;
    for (size_t k = 0; k < nb; ++k) {
        const talp_gpu_raw_batch& b = rb[k];
        if ((b.flags & TALP_GPU_DEVICE_PTRS) != (rb[0].flags & TALP_GPU_DEVICE_PTRS))
            return fail(TALP_GPU_EINVAL, "raw batches mix host and device pointers");
        if (b.flags & ~(TALP_GPU_DEVICE_PTRS | TALP_GPU_APPEND | TALP_GPU_HOLD_BACK))
            return fail(TALP_GPU_EINVAL, "raw: unknown flags");
        if (b.n_ranks == 0 || !b.devices_per_rank || !b.raw_off || !b.host_off)
            return fail(TALP_GPU_EINVAL, "raw: bad header");
        if (b.raw_off[0] != 0) return fail(TALP_GPU_EINVAL, "raw: raw_off[0] != 0");
        for (size_t j = 0; j < k; ++j)
            if (rb[j].trace_id == b.trace_id) return fail(TALP_GPU_EINVAL, "raw: a trace twice in one call");
        hb[k] = (b.flags & TALP_GPU_HOLD_BACK) != 0;
        if (hb[k] && !b.stream_mask) return fail(TALP_GPU_EINVAL, "raw: hold-back needs the stream masks");
        auto it = holds.find(b.trace_id);
        if (it != holds.end() && (b.flags & TALP_GPU_APPEND)) {
            RawHold* h = it->second;
            if (h->n != b.n_ranks || !std::equal(h->dpr.begin(), h->dpr.end(), b.devices_per_rank))
                return fail(TALP_GPU_EINVAL, "raw: shape differs from the held records' trace");
            hs[k] = h;
        }
        outn = align_up(outn, 16);
        out_base[k] = outn;
        uint64_t m = 0, n_in = 0;
        for (uint32_t i = 0; i < b.n_ranks; ++i) {
            const uint32_t D = b.devices_per_rank[i];
            if (D > static_cast<uint32_t>(kRawMaxDevices))
                return fail(TALP_GPU_EINVAL, "raw: more than 8 devices in a rank");
            if (b.raw_off[i + 1] < b.raw_off[i]) return fail(TALP_GPU_EINVAL, "raw: raw_off decreases");
            const uint64_t n = b.raw_off[i + 1] - b.raw_off[i];
            const uint64_t held = hs[k] ? hs[k]->cnt[i] : 0;
            if (n && D == 0) return fail(TALP_GPU_EINVAL, "raw: records of a rank without devices");
            if (hb[k] && n + held >= (1ull << 32)) return fail(TALP_GPU_EINVAL, "raw: 2^32 records in a held rank");
            nt += (held + tile - 1) / tile + (n + tile - 1) / tile;
            n_in += n + held;
            m += D;
        }
        m_of[k] = m;
        mtot += m;
        nrk += b.n_ranks;
        const uint64_t n = b.raw_off[b.n_ranks];
        if (n && (!b.raw_se || !b.raw_tag || !b.raw_dev)) return fail(TALP_GPU_EINVAL, "raw: null record arrays");
        if (dev_ptrs && (reinterpret_cast<uintptr_t>(b.raw_se) & 15u))
            return fail(TALP_GPU_EINVAL, "raw: raw_se not 16-byte aligned");
        nr += n;
        outn += n_in;
        nh = align_up(nh, 16);
        hbase[k] = nh;
        nh += b.host_off[b.n_ranks];
        any_hold = any_hold || hb[k];
    }
    if (nt > 0xFFFFFFFFull || mtot > 0xFFFFFFFFull || nrk > 0xFFFFFFFFull)
        return fail(TALP_GPU_EINVAL, "raw: too large");

    // device buffer: [input staging][host staging][lanes][fold lanes][tables][fold bases][hist][offs][moves]
    //                [device counts][fold counts][hold counts][status]
    size_t o = 0;
    const size_t o_rse = o; o = align_up(o + (dev_ptrs ? 0 : 16 * nr), 256);
    const size_t o_rtag = o; o = align_up(o + (dev_ptrs ? 0 : nr), 256);
    const size_t o_rdev = o; o = align_up(o + (dev_ptrs ? 0 : nr), 256);
    const size_t o_hse = o; o = align_up(o + (dev_ptrs ? 0 : 16 * nh), 256);
    const size_t o_hst = o; o = align_up(o + (dev_ptrs ? 0 : nh + 16), 256);
    const size_t o_lse = o; o = align_up(o + 16 * outn, 256);
    const size_t o_ltag = o; o = align_up(o + outn + 16, 256);
    const size_t o_fse = o; o = align_up(o + (any_hold ? 16 * outn : 0), 256);
    const size_t o_ftag = o; o = align_up(o + (any_hold ? outn + 16 : 0), 256);
    const size_t o_ranks = o; o = align_up(o + sizeof(RawRank) * nrk, 256);
    const size_t o_tiles = o; o = align_up(o + sizeof(RawTile) * nt, 256);
    const size_t tab_bytes = o - o_ranks;
    const size_t o_fbase = o; o = align_up(o + 8 * nrk, 256);
    const size_t o_hist = o; o = align_up(o + 4ull * kRawBuckets * nt, 256);
    const size_t o_offs = o; o = align_up(o + 8ull * kRawBuckets * nt, 256);
    const size_t o_moves = o; o = align_up(o + (any_hold ? sizeof(RawMove) * kRawBuckets * nrk : 0), 256);
    const size_t o_runs = o; o = align_up(o + 8ull * kRunsStride * mtot, 256);
    const size_t o_cnt = o; o = align_up(o + 8 * mtot, 256);
    const size_t o_fcnt = o; o = align_up(o + 8 * mtot, 256);
    const size_t o_hcnt = o; o = align_up(o + 8 * nrk, 256);
    const size_t o_nstr = o; o = align_up(o + 4 * mtot, 256);
    const size_t o_st = o; o += 256;
    const size_t down_bytes = o - o_cnt;

    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    TALP_CUDA(cudaSetDevice(c->device));
    if (c->raw_used) TALP_CUDA(cudaStreamWaitEvent(stream, c->ev_raw, 0));
    TALP_TRY(grow(c, c->raw, o));
    char* R = static_cast<char*>(c->raw.p);

    // hold states: new ones for hold-back batches without one, and the
    // buffer the held records of this call go to
    std::vector<RawHold*> hn(nb, nullptr);
    for (size_t k = 0; k < nb; ++k) {
        if (!hb[k]) continue;
        const talp_gpu_raw_batch& b = rb[k];
        RawHold* h = hs[k];
        if (!h) {
            raw_hold_drop(c, b.trace_id);
            h = new RawHold();
            h->n = b.n_ranks;
            h->dpr.assign(b.devices_per_rank, b.devices_per_rank + b.n_ranks);
            h->off.assign(b.n_ranks, 0);
            h->cnt.assign(b.n_ranks, 0);
            talp_gpu_status st = grow(c, h->ls, sizeof(int64_t) * kRawBuckets * b.n_ranks);
            if (st != TALP_GPU_OK) {
                delete h;
                return st;
            }
            holds[b.trace_id] = h;
        }
        h->smask.assign(b.stream_mask, b.stream_mask + b.n_ranks * kRawMaxDevices);
        uint64_t n_in = b.raw_off[b.n_ranks];
        for (uint64_t v : h->cnt) n_in += v;
        TALP_TRY(grow(c, h->buf[1 - h->cur], hold_bytes(n_in)));
        h->o_tag[1 - h->cur] = hold_tag_at(n_in);
        h->o_dev[1 - h->cur] = hold_dev_at(n_in);
        hn[k] = h;
    }

    // pass 2: ranks and tiles (held records first, then the new ones)
    std::vector<RawRank> ranks;
    std::vector<RawTile> tiles;
    ranks.reserve(nrk);
    tiles.reserve(nt);
    std::vector<std::vector<uint64_t>> slot(nb);   // hold-back: each rank's slot in the next held buffer
    {
        uint64_t p = 0, g0 = 0;
        for (size_t k = 0; k < nb; ++k) {
            const talp_gpu_raw_batch& b = rb[k];
            const int64_t* se = dev_ptrs ? b.raw_se : reinterpret_cast<const int64_t*>(R + o_rse) + 2 * p;
            const uint8_t* tg = dev_ptrs ? b.raw_tag : reinterpret_cast<const uint8_t*>(R + o_rtag) + p;
            const uint8_t* dv = dev_ptrs ? b.raw_dev : reinterpret_cast<const uint8_t*>(R + o_rdev) + p;
            RawHold* h = hs[k];     // held records read
            RawHold* hx = hn[k];    // held records written
            const char* hbuf = h ? static_cast<const char*>(h->buf[h->cur].p) : nullptr;
            char* nbuf = hx ? static_cast<char*>(hx->buf[1 - hx->cur].p) : nullptr;
            slot[k].assign(b.n_ranks, 0);
            uint64_t rel = 0;
            for (uint32_t i = 0; i < b.n_ranks; ++i) {
                RawRank r;
                memset(&r, 0, sizeof(r));
                r.out0 = out_base[k] + rel;
                r.dev0 = static_cast<uint32_t>(g0);
                r.D = b.devices_per_rank[i];
                r.tile0 = static_cast<uint32_t>(tiles.size());
                const uint32_t ri = static_cast<uint32_t>(ranks.size());
                const uint64_t held = h ? h->cnt[i] : 0;
                for (uint64_t q = 0; q < held; q += tile)
                    tiles.push_back(RawTile{reinterpret_cast<const int64_t*>(hbuf) + 2 * (h->off[i] + q),
                                            reinterpret_cast<const uint8_t*>(hbuf + h->o_tag[h->cur]) + h->off[i] + q,
                                            reinterpret_cast<const uint8_t*>(hbuf + h->o_dev[h->cur]) + h->off[i] + q,
                                            r.out0 + q, static_cast<uint32_t>(std::min<uint64_t>(tile, held - q)),
                                            ri});
                const uint64_t n = b.raw_off[i + 1] - b.raw_off[i];
                for (uint64_t q = 0; q < n; q += tile)
                    tiles.push_back(RawTile{se + 2 * (b.raw_off[i] + q), tg + b.raw_off[i] + q, dv + b.raw_off[i] + q,
                                            r.out0 + held + q, static_cast<uint32_t>(std::min<uint64_t>(tile, n - q)),
                                            ri});
                r.ntile = static_cast<uint32_t>(tiles.size()) - r.tile0;
                if (hx) {
                    r.last_start = static_cast<int64_t*>(hx->ls.p) + static_cast<uint64_t>(kRawBuckets) * i;
                    r.hold_se = reinterpret_cast<int64_t*>(nbuf) + 2 * rel;
                    r.hold_tag = reinterpret_cast<uint8_t*>(nbuf + hx->o_tag[1 - hx->cur]) + rel;
                    r.hold_dev = reinterpret_cast<uint8_t*>(nbuf + hx->o_dev[1 - hx->cur]) + rel;
                    for (int d = 0; d < kRawMaxDevices; ++d) r.smask[d] = hx->smask[i * kRawMaxDevices + d];
                    r.fresh = hx->fresh ? 1u : 0u;
                    slot[k][i] = rel;
                }
                ranks.push_back(r);
                rel += held + n;
                g0 += r.D;
            }
            p += b.raw_off[b.n_ranks];
        }
    }

    TALP_CUDA(cudaEventSynchronize(c->ev_up));
    TALP_TRY(grow_pinned(c->up, tab_bytes + 8 * nrk));
    memcpy(c->up.p, ranks.data(), sizeof(RawRank) * nrk);
    if (nt) memcpy(static_cast<char*>(c->up.p) + (o_tiles - o_ranks), tiles.data(), sizeof(RawTile) * nt);
    TALP_CUDA(cudaMemcpyAsync(R + o_ranks, c->up.p, tab_bytes, cudaMemcpyHostToDevice, stream));
    TALP_CUDA(cudaEventRecord(c->ev_up, stream));
    if (!dev_ptrs) {
        uint64_t p = 0;
        for (size_t k = 0; k < nb; ++k) {
            const uint64_t n = rb[k].raw_off[rb[k].n_ranks];
            if (n) {
                TALP_CUDA(cudaMemcpyAsync(R + o_rse + 16 * p, rb[k].raw_se, 16 * n, cudaMemcpyHostToDevice, stream));
                TALP_CUDA(cudaMemcpyAsync(R + o_rtag + p, rb[k].raw_tag, n, cudaMemcpyHostToDevice, stream));
                TALP_CUDA(cudaMemcpyAsync(R + o_rdev + p, rb[k].raw_dev, n, cudaMemcpyHostToDevice, stream));
            }
            const uint64_t h = rb[k].host_off[rb[k].n_ranks];
            if (h) {
                if (!rb[k].host_se || !rb[k].host_state) return fail(TALP_GPU_EINVAL, "raw: null host arrays");
                TALP_CUDA(cudaMemcpyAsync(R + o_hse + 16 * hbase[k], rb[k].host_se, 16 * h, cudaMemcpyHostToDevice,
                                          stream));
                TALP_CUDA(cudaMemcpyAsync(R + o_hst + hbase[k], rb[k].host_state, h, cudaMemcpyHostToDevice, stream));
            }
            p += n;
        }
    }
    TALP_CUDA(cudaMemsetAsync(R + o_st, 0, 16, stream));
    const int grid = static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(nt, static_cast<uint64_t>(c->num_sms) * 8)));
    const RawTile* dtiles = reinterpret_cast<const RawTile*>(R + o_tiles);
    const RawRank* dranks = reinterpret_cast<const RawRank*>(R + o_ranks);
    RawMove* dmoves = any_hold ? reinterpret_cast<RawMove*>(R + o_moves) : nullptr;
    uint32_t* dst = reinterpret_cast<uint32_t*>(R + o_st);
    TALP_CUDA(launch_raw_count(dtiles, static_cast<uint32_t>(nt), dranks, static_cast<uint32_t>(nrk),
                               reinterpret_cast<uint32_t*>(R + o_hist), reinterpret_cast<uint64_t*>(R + o_offs), dmoves,
                               reinterpret_cast<uint64_t*>(R + o_cnt), reinterpret_cast<uint32_t*>(R + o_nstr),
                               reinterpret_cast<uint64_t*>(R + o_runs), dst,
                               grid, stream));
    TALP_CUDA(launch_raw_scatter(dtiles, static_cast<uint32_t>(nt), dranks, reinterpret_cast<const uint64_t*>(R + o_offs),
                                 reinterpret_cast<int64_t*>(R + o_lse), reinterpret_cast<uint8_t*>(R + o_ltag), dst,
                                 c->wait_limit, grid, stream));
    c->kernel_launches += (nt ? 2 : 0) + (nrk ? 1 : 0);
    if (any_hold) {
        TALP_CUDA(launch_raw_hold(dranks, static_cast<uint32_t>(nrk), reinterpret_cast<const int64_t*>(R + o_lse), dmoves,
                                  reinterpret_cast<uint64_t*>(R + o_fcnt), reinterpret_cast<uint64_t*>(R + o_hcnt), dst,
                                  reinterpret_cast<uint64_t*>(R + o_runs),
                                  stream));
        ++c->kernel_launches;
    }
    // the ingest needs each device's record count on the host
    TALP_TRY(grow_pinned(c->down, down_bytes));
    TALP_CUDA(cudaMemcpyAsync(c->down.p, R + o_cnt, down_bytes, cudaMemcpyDeviceToHost, stream));
    TALP_CUDA(cudaStreamSynchronize(stream));
    const char* D = static_cast<const char*>(c->down.p);
    const uint64_t* cnt = reinterpret_cast<const uint64_t*>(D);
    const uint64_t* fcnt = reinterpret_cast<const uint64_t*>(D + (o_fcnt - o_cnt));
    const uint64_t* hcnt = reinterpret_cast<const uint64_t*>(D + (o_hcnt - o_cnt));
    const uint32_t* nstr = reinterpret_cast<const uint32_t*>(D + (o_nstr - o_cnt));
    uint32_t status = 0;
    memcpy(&status, D + (o_st - o_cnt), 4);
    if (status) {
        for (size_t k = 0; k < nb; ++k)
            if (hb[k]) raw_hold_drop(c, rb[k].trace_id);
        if (status & ST_TIMEOUT) return fail(TALP_GPU_ETIMEDOUT, "raw: a device-side wait ran out");
        if (status & 1u) return fail(TALP_GPU_EINVAL, "raw: a record names a device its rank does not have");
        return fail(TALP_GPU_EINVAL, "raw: a record on a stream its device's stream mask does not declare");
    }

    std::vector<std::vector<uint64_t>> dev_off(nb);
    std::vector<talp_gpu_trace_batch> tb(nb);
    uint64_t* fbase = static_cast<uint64_t*>(c->up.p) + tab_bytes / 8;   // the table upload has completed
    uint64_t g = 0, ri = 0;
    // a device whose lane is several non-empty streams is out of start order
    // unless its streams happen not to interleave: it skips the first sweep
    // (the sort stage finds and keeps a lane that is in order after all).
    // With hold-back the fold lane holds a part of those streams.
    c->raw_presort.assign(mtot, 0);
    for (size_t k = 0; k < nb; ++k) {
        const talp_gpu_raw_batch& b = rb[k];
        const uint64_t* cn = hb[k] ? fcnt : cnt;
        dev_off[k].assign(m_of[k] + 1, 0);
        for (uint64_t d = 0; d < m_of[k]; ++d, ++g) {
            dev_off[k][d + 1] = dev_off[k][d] + cn[g];
            c->raw_presort[g] = nstr[g] > 1 ? 1 : 0;
        }
        uint64_t dl = 0;   // first device of rank i within the batch
        for (uint32_t i = 0; i < b.n_ranks; ++i, ++ri) {
            fbase[ri] = out_base[k] + dev_off[k][dl];
            dl += b.devices_per_rank[i];
        }
        talp_gpu_trace_batch& t = tb[k];
        memset(&t, 0, sizeof(t));
        t.trace_id = b.trace_id;
        t.n_ranks = b.n_ranks;
        t.n_regions = b.n_regions;
        t.flags = TALP_GPU_DEVICE_PTRS | (b.flags & TALP_GPU_APPEND);
        t.devices_per_rank = b.devices_per_rank;
        t.region_window = b.region_window;
        t.host_se = dev_ptrs ? b.host_se : reinterpret_cast<const int64_t*>(R + o_hse) + 2 * hbase[k];
        t.host_state = dev_ptrs ? b.host_state : reinterpret_cast<const uint8_t*>(R + o_hst) + hbase[k];
        t.host_off = b.host_off;
        const size_t lo = hb[k] ? o_fse : o_lse, lt = hb[k] ? o_ftag : o_ltag;
        t.dev_se = reinterpret_cast<const int64_t*>(R + lo) + 2 * out_base[k];
        t.dev_tag = reinterpret_cast<const uint8_t*>(R + lt) + out_base[k];
        t.dev_off = dev_off[k].data();
    }
    if (any_hold) {
        TALP_CUDA(cudaMemcpyAsync(R + o_fbase, fbase, 8 * nrk, cudaMemcpyHostToDevice, stream));
        TALP_CUDA(cudaEventRecord(c->ev_up, stream));
        TALP_CUDA(launch_raw_move(dtiles, static_cast<uint32_t>(nt), dranks, dmoves,
                                  reinterpret_cast<const uint64_t*>(R + o_fbase),
                                  reinterpret_cast<const int64_t*>(R + o_lse), reinterpret_cast<const uint8_t*>(R + o_ltag),
                                  reinterpret_cast<int64_t*>(R + o_fse), reinterpret_cast<uint8_t*>(R + o_ftag), grid,
                                  stream));
        ++c->kernel_launches;
        ri = 0;
        for (size_t k = 0; k < nb; ++k) {
            if (!hb[k]) {
                ri += rb[k].n_ranks;
                continue;
            }
            RawHold* h = hn[k];
            for (uint32_t i = 0; i < rb[k].n_ranks; ++i, ++ri) {
                h->off[i] = slot[k][i];
                h->cnt[i] = hcnt[ri];
            }
            h->cur = 1 - h->cur;
            h->fresh = false;
        }
    }
    // a batch without hold-back folded every held record: its hold state ends
    for (size_t k = 0; k < nb; ++k)
        if (!hb[k] && holds.count(rb[k].trace_id)) raw_hold_drop(c, rb[k].trace_id);
    c->raw_inner = true;
    c->raw_runs = reinterpret_cast<const uint64_t*>(R + o_runs);
    const talp_gpu_status st = talp_gpu_ingest_events(c, tb.data(), nb, stream_);
    c->raw_inner = false;
    c->raw_runs = nullptr;
    c->raw_presort.clear();
    TALP_CUDA(cudaEventRecord(c->ev_raw, stream));
    c->raw_used = true;
    return st;
}

static talp_gpu_status thread_tree_common(talp_gpu_ctx* c, uint64_t trace_id, uint32_t region,
                                          const uint32_t* proc_off, uint32_t n_procs, ThreadOut* out_dev_user,
                                          talp_gpu_thread_tree* out_host, cudaStream_t stream) {
    static_assert(sizeof(ThreadOut) == sizeof(talp_gpu_thread_tree), "thread tree record layout");
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    if (!proc_off || (!out_host && !out_dev_user)) return fail(TALP_GPU_EINVAL, "null argument");
    if (n_procs == 0) return fail(TALP_GPU_EINVAL, "no processes");
    auto it = c->traces.find(trace_id);
    if (it == c->traces.end()) return fail(TALP_GPU_ENOTFOUND, "unknown trace id " + std::to_string(trace_id));
    TraceState* t = it->second;
    if (proc_off[0] != 0 || proc_off[n_procs] != t->n)
        return fail(TALP_GPU_EINVAL, "proc_off must run from 0 to the trace's n_ranks");
    for (uint32_t i = 0; i < n_procs; ++i)
        if (proc_off[i + 1] <= proc_off[i]) return fail(TALP_GPU_EINVAL, "a process without threads in proc_off");
    std::vector<uint32_t> regions;
    if (region == TALP_GPU_ALL_REGIONS) {
        for (uint32_t r = 0; r < t->R; ++r) regions.push_back(r);
    } else {
        if (region >= t->R) return fail(TALP_GPU_EINVAL, "region out of range");
        regions.push_back(region);
    }
    TALP_CUDA(cudaSetDevice(c->device));
    const size_t nj = regions.size();
    const size_t jb = align_up(sizeof(ThreadJob) * nj, 256);
    const size_t pbytes = sizeof(uint32_t) * (static_cast<size_t>(n_procs) + 1);
    const size_t ob = align_up(jb + pbytes, 256);
    if (c->ws_used) TALP_CUDA(cudaStreamWaitEvent(stream, c->ev_ws, 0));
    TALP_TRY(grow(c, c->ws, ob + sizeof(ThreadOut) * nj));
    char* ws = static_cast<char*>(c->ws.p);
    const uint32_t* dpo = reinterpret_cast<const uint32_t*>(ws + jb);
    ThreadOut* res = reinterpret_cast<ThreadOut*>(ws + ob);
    ThreadOut* dout = out_dev_user ? out_dev_user : res;
    TALP_CUDA(cudaEventSynchronize(c->ev_upf));
    TALP_TRY(grow_pinned(c->upf, jb + pbytes));
    char* up = static_cast<char*>(c->upf.p);
    for (size_t k = 0; k < nj; ++k)
        reinterpret_cast<ThreadJob*>(up)[k] = ThreadJob{t->tdev, dout + k, dpo, n_procs, regions[k]};
    memcpy(up + jb, proc_off, pbytes);
    TALP_CUDA(cudaMemcpyAsync(ws, up, jb + pbytes, cudaMemcpyHostToDevice, stream));
    TALP_CUDA(cudaEventRecord(c->ev_upf, stream));
    TALP_CUDA(launch_thread_tree(reinterpret_cast<const ThreadJob*>(ws), static_cast<uint32_t>(nj), stream));
    ++c->kernel_launches;
    if (out_dev_user) {
        TALP_CUDA(cudaEventRecord(c->ev_ws, stream));
        c->ws_used = true;
        return TALP_GPU_OK;
    }
    TALP_TRY(grow_pinned(c->down, sizeof(ThreadOut) * nj));
    TALP_CUDA(cudaMemcpyAsync(c->down.p, res, sizeof(ThreadOut) * nj, cudaMemcpyDeviceToHost, stream));
    TALP_CUDA(cudaEventRecord(c->ev_ws, stream));
    c->ws_used = true;
    TALP_CUDA(cudaStreamSynchronize(stream));
    memcpy(out_host, c->down.p, sizeof(ThreadOut) * nj);
    for (size_t k = 0; k < nj; ++k) {
        const uint32_t f = out_host[k].flags;
        if (f & TALP_GPU_M_TIMEOUT) return fail(TALP_GPU_ETIMEDOUT, "a device-side wait ran out during ingest");
        if (f & (TALP_GPU_M_INVALID | TALP_GPU_M_UNSORTED))
            return fail(TALP_GPU_EINVAL, "invalid or out-of-order records were ingested");
    }
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_thread_metrics(talp_gpu_ctx* c, uint64_t trace_id, uint32_t region,
                                        const uint32_t* proc_off, uint32_t n_procs,
                                        talp_gpu_thread_tree* out_host, void* stream) {
    if (!out_host) return fail(TALP_GPU_EINVAL, "null out");
    return thread_tree_common(c, trace_id, region, proc_off, n_procs, nullptr, out_host,
                              static_cast<cudaStream_t>(stream));
}

talp_gpu_status talp_gpu_thread_metrics_device(talp_gpu_ctx* c, uint64_t trace_id, uint32_t region,
                                               const uint32_t* proc_off, uint32_t n_procs,
                                               talp_gpu_thread_tree* out_device, void* stream) {
    if (!out_device) return fail(TALP_GPU_EINVAL, "null out");
    if ((reinterpret_cast<uintptr_t>(out_device) & 7u) != 0) return fail(TALP_GPU_EINVAL, "out_device misaligned");
    return thread_tree_common(c, trace_id, region, proc_off, n_procs, reinterpret_cast<ThreadOut*>(out_device),
                              nullptr, static_cast<cudaStream_t>(stream));
}

talp_gpu_status talp_gpu_thread_metrics_combine(talp_gpu_ctx* c, const talp_gpu_thread_tree* parts, size_t n_parts,
                                                talp_gpu_thread_tree* out_host, void* stream_) {
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    if (!parts || !out_host || n_parts == 0) return fail(TALP_GPU_EINVAL, "null argument or no parts");
    if (n_parts > (1u << 20)) return fail(TALP_GPU_EINVAL, "more than 2^20 parts");
    for (size_t k = 1; k < n_parts; ++k)
        if (parts[k].trace_id != parts[0].trace_id || parts[k].region != parts[0].region)
            return fail(TALP_GPU_EINVAL, "parts of different traces or regions");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    TALP_CUDA(cudaSetDevice(c->device));
    const size_t pb = align_up(sizeof(ThreadOut) * n_parts, 256);
    if (c->ws_used) TALP_CUDA(cudaStreamWaitEvent(stream, c->ev_ws, 0));
    TALP_TRY(grow(c, c->ws, pb + sizeof(ThreadOut)));
    ThreadOut* dparts = static_cast<ThreadOut*>(c->ws.p);
    ThreadOut* dres = reinterpret_cast<ThreadOut*>(static_cast<char*>(c->ws.p) + pb);
    TALP_CUDA(cudaEventSynchronize(c->ev_up));
    TALP_TRY(grow_pinned(c->up, pb));
    memcpy(c->up.p, parts, sizeof(ThreadOut) * n_parts);
    TALP_CUDA(cudaMemcpyAsync(dparts, c->up.p, sizeof(ThreadOut) * n_parts, cudaMemcpyHostToDevice, stream));
    TALP_CUDA(cudaEventRecord(c->ev_up, stream));
    TALP_CUDA(launch_thread_combine(dparts, static_cast<uint32_t>(n_parts), dres, stream));
    ++c->kernel_launches;
    TALP_TRY(grow_pinned(c->down, sizeof(ThreadOut)));
    TALP_CUDA(cudaMemcpyAsync(c->down.p, dres, sizeof(ThreadOut), cudaMemcpyDeviceToHost, stream));
    TALP_CUDA(cudaEventRecord(c->ev_ws, stream));
    c->ws_used = true;
    TALP_CUDA(cudaStreamSynchronize(stream));
    memcpy(out_host, c->down.p, sizeof(ThreadOut));
    const uint32_t f = out_host->flags;
    if (f & TALP_GPU_M_TIMEOUT) return fail(TALP_GPU_ETIMEDOUT, "a device-side wait ran out during ingest");
    if (f & (TALP_GPU_M_INVALID | TALP_GPU_M_UNSORTED))
        return fail(TALP_GPU_EINVAL, "invalid or out-of-order records were ingested");
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_scalability(talp_gpu_ctx* c, const talp_gpu_metrics* runs, size_t n_runs, size_t ref,
                                     uint32_t mode, talp_gpu_scaling* out_host, void* stream_) {
    static_assert(sizeof(ScaleOut) == sizeof(talp_gpu_scaling), "scaling record layout");
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    if (!runs || !out_host || n_runs == 0) return fail(TALP_GPU_EINVAL, "null argument or no runs");
    if (n_runs > (1u << 20)) return fail(TALP_GPU_EINVAL, "more than 2^20 runs");
    if (ref >= n_runs) return fail(TALP_GPU_EINVAL, "reference run out of range");
    if (mode != TALP_GPU_SCALING_STRONG && mode != TALP_GPU_SCALING_WEAK) return fail(TALP_GPU_EINVAL, "bad mode");
    for (size_t k = 1; k < n_runs; ++k)
        if (runs[k].region != runs[0].region) return fail(TALP_GPU_EINVAL, "runs of different regions");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    TALP_CUDA(cudaSetDevice(c->device));
    const size_t rb = align_up(sizeof(MetricsOut) * n_runs, 256);
    if (c->ws_used) TALP_CUDA(cudaStreamWaitEvent(stream, c->ev_ws, 0));
    TALP_TRY(grow(c, c->ws, rb + sizeof(ScaleOut) * n_runs));
    MetricsOut* druns = static_cast<MetricsOut*>(c->ws.p);
    ScaleOut* dout = reinterpret_cast<ScaleOut*>(static_cast<char*>(c->ws.p) + rb);
    TALP_CUDA(cudaEventSynchronize(c->ev_up));
    TALP_TRY(grow_pinned(c->up, rb));
    memcpy(c->up.p, runs, sizeof(MetricsOut) * n_runs);
    TALP_CUDA(cudaMemcpyAsync(druns, c->up.p, sizeof(MetricsOut) * n_runs, cudaMemcpyHostToDevice, stream));
    TALP_CUDA(cudaEventRecord(c->ev_up, stream));
    TALP_CUDA(launch_scalability(druns, static_cast<uint32_t>(n_runs), static_cast<uint32_t>(ref),
                                 mode == TALP_GPU_SCALING_WEAK ? 1 : 0, dout, stream));
    ++c->kernel_launches;
    TALP_TRY(grow_pinned(c->down, sizeof(ScaleOut) * n_runs));
    TALP_CUDA(cudaMemcpyAsync(c->down.p, dout, sizeof(ScaleOut) * n_runs, cudaMemcpyDeviceToHost, stream));
    TALP_CUDA(cudaEventRecord(c->ev_ws, stream));
    c->ws_used = true;
    TALP_CUDA(cudaStreamSynchronize(stream));
    memcpy(out_host, c->down.p, sizeof(ScaleOut) * n_runs);
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_concurrency(talp_gpu_ctx* c, const talp_gpu_trace_batch* b, uint32_t region,
                                     int64_t* out_host, void* stream_) {
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    if (!b || !out_host) return fail(TALP_GPU_EINVAL, "null argument");
    if (b->n_ranks == 0 || !b->devices_per_rank || !b->region_window || !b->dev_off)
        return fail(TALP_GPU_EINVAL, "concurrency: bad header");
    if (region >= b->n_regions || b->n_regions > TALP_GPU_MAX_REGIONS)
        return fail(TALP_GPU_EINVAL, "concurrency: region out of range");
    uint64_t m = 0;
    for (uint32_t i = 0; i < b->n_ranks; ++i) m += b->devices_per_rank[i];
    if (m == 0) return TALP_GPU_OK;
    if (m > (1u << 24)) return fail(TALP_GPU_EINVAL, "concurrency: too many devices");
    if (b->dev_off[0] != 0) return fail(TALP_GPU_EINVAL, "concurrency: dev_off[0] != 0");
    for (uint64_t g = 0; g < m; ++g)
        if (b->dev_off[g + 1] < b->dev_off[g]) return fail(TALP_GPU_EINVAL, "concurrency: dev_off decreases");
    const uint64_t N = b->dev_off[m];
    const bool dev_ptrs = (b->flags & TALP_GPU_DEVICE_PTRS) != 0;
    if (N && (!b->dev_se || !b->dev_tag)) return fail(TALP_GPU_EINVAL, "concurrency: null record arrays");
    if (N && dev_ptrs && (reinterpret_cast<uintptr_t>(b->dev_se) & 15u))
        return fail(TALP_GPU_EINVAL, "concurrency: dev_se not 16-byte aligned");

    // device and chunk tables (chunks of at most kChunk records)
    constexpr uint64_t kChunk = 16384;
    std::vector<ConcDev> devs(m);
    std::vector<ConcChunk> chunks;
    uint64_t g = 0;
    for (uint32_t i = 0; i < b->n_ranks; ++i) {
        const int64_t* w = b->region_window + (static_cast<uint64_t>(region) * b->n_ranks + i) * 2;
        for (uint32_t d = 0; d < b->devices_per_rank[i]; ++d, ++g) {
            ConcDev& v = devs[g];
            v.a = w[0];
            v.b = w[1];
            v.rec0 = b->dev_off[g];
            v.n = b->dev_off[g + 1] - b->dev_off[g];
            v.chunk0 = static_cast<uint32_t>(chunks.size());
            for (uint64_t o = 0; o < v.n; o += kChunk)
                chunks.push_back(ConcChunk{v.rec0 + o, static_cast<uint32_t>(std::min(kChunk, v.n - o)),
                                           static_cast<uint32_t>(g)});
            v.nchunk = static_cast<uint32_t>(chunks.size()) - v.chunk0;
        }
    }
    const size_t nc = chunks.size();
    const size_t o_dev = 0;
    const size_t o_chunk = align_up(o_dev + sizeof(ConcDev) * m, 256);
    const size_t o_top = align_up(o_chunk + sizeof(ConcChunk) * nc, 256);
    const size_t o_in = align_up(o_top + sizeof(int64_t) * 2 * kConcLevels * nc, 256);
    const size_t o_snap = align_up(o_in + sizeof(int64_t) * 2 * kConcLevels * nc, 256);
    const size_t o_out = align_up(o_snap + sizeof(int64_t) * 2 * 2 * kConcLevels * nc, 256);
    const size_t o_st = align_up(o_out + sizeof(int64_t) * 2 * kConcLevels * m, 256);
    const size_t ws_bytes = o_st + 256;
    const size_t up_bytes = o_top;
    const size_t down_bytes = o_st + 16 - o_out;
    const size_t stage_bytes = dev_ptrs ? 0 : align_up(16 * N, 256) + align_up(N + 16, 256);

    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    TALP_CUDA(cudaSetDevice(c->device));
    if (c->ws_used) TALP_CUDA(cudaStreamWaitEvent(stream, c->ev_ws, 0));
    TALP_TRY(grow(c, c->ws, ws_bytes));
    if (stage_bytes) TALP_TRY(grow(c, c->stage, stage_bytes));
    TALP_CUDA(cudaEventSynchronize(c->ev_up));
    TALP_TRY(grow_pinned(c->up, up_bytes));
    TALP_TRY(grow_pinned(c->down, down_bytes));
    char* up = static_cast<char*>(c->up.p);
    memcpy(up + o_dev, devs.data(), sizeof(ConcDev) * m);
    if (nc) memcpy(up + o_chunk, chunks.data(), sizeof(ConcChunk) * nc);
    char* ws = static_cast<char*>(c->ws.p);
    TALP_CUDA(cudaMemcpyAsync(ws, up, up_bytes, cudaMemcpyHostToDevice, stream));
    TALP_CUDA(cudaEventRecord(c->ev_up, stream));
    const int64_t* se = b->dev_se;
    const uint8_t* tag = b->dev_tag;
    if (!dev_ptrs && N) {
        char* st = static_cast<char*>(c->stage.p);
        TALP_CUDA(cudaMemcpyAsync(st, b->dev_se, 16 * N, cudaMemcpyHostToDevice, stream));
        TALP_CUDA(cudaMemcpyAsync(st + align_up(16 * N, 256), b->dev_tag, N, cudaMemcpyHostToDevice, stream));
        se = reinterpret_cast<const int64_t*>(st);
        tag = reinterpret_cast<const uint8_t*>(st + align_up(16 * N, 256));
    }
    TALP_CUDA(cudaMemsetAsync(ws + o_out, 0, o_st + 16 - o_out, stream));
    TALP_CUDA(launch_concurrency(se, tag, reinterpret_cast<const ConcDev*>(ws + o_dev), static_cast<uint32_t>(m),
                                 reinterpret_cast<const ConcChunk*>(ws + o_chunk), static_cast<uint32_t>(nc),
                                 reinterpret_cast<int64_t*>(ws + o_top), reinterpret_cast<int64_t*>(ws + o_in),
                                 reinterpret_cast<int64_t*>(ws + o_snap),
                                 reinterpret_cast<int64_t*>(ws + o_out), reinterpret_cast<uint32_t*>(ws + o_st),
                                 stream));
    c->kernel_launches += nc ? 3 : 0;
    TALP_CUDA(cudaMemcpyAsync(c->down.p, ws + o_out, down_bytes, cudaMemcpyDeviceToHost, stream));
    TALP_CUDA(cudaEventRecord(c->ev_ws, stream));
    c->ws_used = true;
    TALP_CUDA(cudaStreamSynchronize(stream));
    memcpy(out_host, c->down.p, sizeof(int64_t) * 2 * kConcLevels * m);
    uint32_t status = 0;
    memcpy(&status, static_cast<char*>(c->down.p) + (o_st - o_out), sizeof(status));
    if (status & 3u) return fail(TALP_GPU_EINVAL, "concurrency: invalid record (end < start or bad kind)");
    if (status & 4u) return fail(TALP_GPU_EINVAL, "concurrency: device records out of start order");
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_unit_sums(talp_gpu_ctx* c, uint64_t trace_id, uint32_t region, int64_t* host_out,
                                   int64_t* dev_out, void* stream_) {
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    auto it = c->traces.find(trace_id);
    if (it == c->traces.end()) return fail(TALP_GPU_ENOTFOUND, "unknown trace id");
    TraceState* t = it->second;
    if (region >= t->R) return fail(TALP_GPU_EINVAL, "region out of range");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    TALP_CUDA(cudaSetDevice(c->device));
    const size_t pitch = sizeof(int64_t) * 3 * t->R;
    if (host_out && t->n)
        TALP_CUDA(cudaMemcpy2DAsync(host_out, 3 * sizeof(int64_t), t->hsum + 3 * region, pitch, 3 * sizeof(int64_t),
                                    t->n, cudaMemcpyDeviceToHost, stream));
    if (dev_out && t->m)
        TALP_CUDA(cudaMemcpy2DAsync(dev_out, 3 * sizeof(int64_t), t->dsum + 3 * region, pitch, 3 * sizeof(int64_t),
                                    t->m, cudaMemcpyDeviceToHost, stream));
    TALP_CUDA(cudaStreamSynchronize(stream));
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_reset(talp_gpu_ctx* c, uint64_t trace_id) {
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    TALP_CUDA(cudaSetDevice(c->device));
    TALP_CUDA(cudaDeviceSynchronize());
    if (trace_id == TALP_GPU_ALL) {
        for (auto& kv : c->traces)
            if (kv.second->plan_refs) return fail(TALP_GPU_EBUSY, "a plan uses one of the traces");
        raw_hold_drop(c, TALP_GPU_ALL);
        for (auto& kv : c->traces) free_trace(c, kv.second);
        c->traces.clear();
        return TALP_GPU_OK;
    }
    auto it = c->traces.find(trace_id);
    if (it == c->traces.end()) return fail(TALP_GPU_ENOTFOUND, "unknown trace id");
    if (it->second->plan_refs) return fail(TALP_GPU_EBUSY, "a plan uses this trace");
    raw_hold_drop(c, trace_id);
    free_trace(c, it->second);
    c->traces.erase(it);
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_profile(talp_gpu_ctx* c, int enable) {
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    c->profiling = enable != 0;
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_profile_read(talp_gpu_ctx* c, talp_gpu_profile_stats* out) {
    if (!c || !out) return fail(TALP_GPU_EINVAL, "null argument");
    TALP_CUDA(cudaSetDevice(c->device));
    out->sweep_launches = c->ev_pending.size();
    out->sweep_records = 0;
    out->sweep_ms = 0.0;
    for (size_t k = 0; k < c->ev_pending.size(); ++k) {
        auto& pr = c->ev_pending[k];
        TALP_CUDA(cudaEventSynchronize(pr.second));
        float ms = 0.f;
        TALP_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
        out->sweep_ms += ms;
        out->sweep_records += c->ev_records[k];
        c->ev_pool.push_back(pr.first);
        c->ev_pool.push_back(pr.second);
    }
    c->ev_pending.clear();
    c->ev_records.clear();
    out->sort_launches = c->sort_ev_pending.size();
    out->sort_ms = 0.0;
    for (auto& pr : c->sort_ev_pending) {
        TALP_CUDA(cudaEventSynchronize(pr.second));
        float ms = 0.f;
        TALP_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
        out->sort_ms += ms;
        c->ev_pool.push_back(pr.first);
        c->ev_pool.push_back(pr.second);
    }
    c->sort_ev_pending.clear();
    out->kernel_launches = c->kernel_launches;
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_memory(talp_gpu_ctx* c, size_t* held, size_t* budget) {
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    if (held) *held = c->held;
    if (budget) *budget = c->budget;
    return TALP_GPU_OK;
}

// ------------------------------------------------------------------- plans

static void plan_release(talp_gpu_plan* p) {
    if (!p) return;
    talp_gpu_ctx* c = p->c;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (TraceState* t : p->ts)
        if (t) --t->plan_refs;
    dev_free(c, p->ws.p, p->ws.cap);
    dev_free(c, p->sortbuf.p, p->sortbuf.cap);
    if (p->up.p) cudaFreeHost(p->up.p);
    --c->dependents;
    delete p;
}

talp_gpu_status talp_gpu_plan_create(talp_gpu_ctx* c, const talp_gpu_trace_batch* batches, size_t nb,
                                     uint32_t plan_flags, talp_gpu_plan** out) {
    if (!c || !out || (nb && !batches)) return fail(TALP_GPU_EINVAL, "null argument");
    *out = nullptr;
    if (nb == 0) return fail(TALP_GPU_EINVAL, "a plan needs at least one trace");
    if (plan_flags & ~TALP_GPU_PLAN_AUTOTUNE) return fail(TALP_GPU_EINVAL, "unknown plan flag bits");
    for (size_t k = 0; k < nb; ++k) {
        if (!(batches[k].flags & TALP_GPU_DEVICE_PTRS) || (batches[k].flags & TALP_GPU_APPEND))
            return fail(TALP_GPU_EINVAL, "a plan takes device-resident records and no APPEND");
    }
    TALP_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = c->cap_stream;

    // candidate tunings (all sized first, so admission sees the largest):
    // every sweep shape x segment costs {1/4, 1, 4} of the default x fixed
    // slices or 16 slices per warp handed out as warps come free
    std::vector<Tuning> cand;
    const Tuning base = pick_tuning(c, batches, nb);
    if ((plan_flags & TALP_GPU_PLAN_AUTOTUNE) && !c->shape_forced) {
        for (int sh = 0; sh < kNumSweepShapes; ++sh)
            for (uint64_t mul : {1ull, 4ull, 16ull})
                for (int spw : {0, 16}) {
                    Tuning t = base;
                    t.shape = sh;
                    t.seg_cost = base.seg_cost * mul / 4;
                    t.spw = spw;
                    cand.push_back(t);
                }
    } else {
        cand.push_back(base);
    }
    std::vector<Layout> Ls(cand.size());
    size_t ws_max = 0, up_max = 0, sb_max = 0;
    for (size_t q = 0; q < cand.size(); ++q) {
        TALP_TRY(size_ingest(c, batches, nb, cand[q], true, Ls[q]));
        ws_max = std::max(ws_max, Ls[q].ws_bytes);
        up_max = std::max(up_max, Ls[q].up_bytes);
        sb_max = std::max(sb_max, Ls[q].sortbuf_bytes);
    }
    const size_t extra = Ls[0].new_bytes + grow_size(ws_max) + (sb_max ? grow_size(sb_max) : 0);
    if (c->held + extra > c->budget)
        return fail(TALP_GPU_ENOMEM, "admission: the plan needs " + std::to_string(extra) +
                                         " more device bytes than the budget leaves");
    if (c->ws_used) TALP_CUDA(cudaStreamWaitEvent(s, c->ev_ws, 0));

    talp_gpu_plan* p = new talp_gpu_plan();
    p->c = c;
    ++c->dependents;
    talp_gpu_status st = get_traces(c, batches, nb, s, p->ts);
    if (st == TALP_GPU_OK) st = grow(c, p->ws, ws_max);
    if (st == TALP_GPU_OK && sb_max) st = grow(c, p->sortbuf, sb_max);
    if (st == TALP_GPU_OK) st = grow_pinned(p->up, up_max);
    if (st != TALP_GPU_OK) {
        plan_release(p);
        return st;
    }
    for (TraceState* t : p->ts) ++t->plan_refs;
    char* up = static_cast<char*>(p->up.p);
    char* wsd = static_cast<char*>(p->ws.p);

    // autotune: time each candidate's launch sequence
    size_t best = 0;
    if (cand.size() > 1) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best_ms = 1e30f;
        for (size_t q = 0; q < cand.size() && st == TALP_GPU_OK; ++q) {
            st = fill_ingest(c, batches, nb, Ls[q], p->ts, up, wsd, nullptr, static_cast<char*>(p->sortbuf.p), s);
            for (int it = 0; it < 4 && st == TALP_GPU_OK; ++it) {   // 1 warm-up (with upload), 3 timed
                if (it == 1) cudaEventRecord(e0, s);
                st = enqueue_ingest(c, Ls[q], up, wsd, s, false, nullptr, it == 0);
            }
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = q;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st != TALP_GPU_OK) {
            plan_release(p);
            return st;
        }
        const Layout& B = Ls[best];
        c->tune[size_class(B.n_records, B.n_segs, B.sorting)] = cand[best];
    }
    p->L = Ls[best];
    p->n_metrics = p->L.n_fin;

    // The tables do not change between launches: upload them once, then
    // capture the kernels (every launch re-initialises what they write).
    st = fill_ingest(c, batches, nb, p->L, p->ts, up, wsd, nullptr, static_cast<char*>(p->sortbuf.p), s);
    if (st == TALP_GPU_OK) {
        cudaError_t e = cudaMemcpyAsync(wsd, up, p->L.up_bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamBeginCapture");
    }
    if (st == TALP_GPU_OK) {
        talp_gpu_status st2 = enqueue_ingest(c, p->L, up, wsd, s, false, &p->launches_per_run, false);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st2 != TALP_GPU_OK) {
            if (g) cudaGraphDestroy(g);
            st = st2;
        } else if (e != cudaSuccess) {
            st = cuda_fail(e, "cudaStreamEndCapture");
        } else {
            p->graph = g;
            e = cudaGraphInstantiate(&p->exec, g, 0);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    if (st != TALP_GPU_OK) {
        plan_release(p);
        return st;
    }
    // after a launch the carries of these traces are in carry[cur ^ 1]
    for (TraceState* t : p->ts) t->cur ^= 1;
    *out = p;
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_plan_launch(talp_gpu_plan* p, void* stream) {
    if (!p) return fail(TALP_GPU_EINVAL, "null plan");
    TALP_CUDA(cudaSetDevice(p->c->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->c->ws_used) TALP_CUDA(cudaStreamWaitEvent(s, p->c->ev_ws, 0));
    TALP_CUDA(cudaGraphLaunch(p->exec, s));
    p->c->kernel_launches += p->launches_per_run;
    TALP_CUDA(cudaEventRecord(p->c->ev_ws, s));
    p->c->ws_used = true;
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_plan_metrics(talp_gpu_plan* p, talp_gpu_metrics* out_host, void* stream) {
    if (!p || !out_host) return fail(TALP_GPU_EINVAL, "null argument");
    TALP_CUDA(cudaSetDevice(p->c->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const MetricsOut* mout = reinterpret_cast<const MetricsOut*>(static_cast<char*>(p->ws.p) + p->L.off_mout);
    TALP_CUDA(cudaMemcpyAsync(out_host, mout, sizeof(MetricsOut) * p->n_metrics, cudaMemcpyDeviceToHost, s));
    TALP_CUDA(cudaStreamSynchronize(s));
    return check_metrics_flags(out_host, p->n_metrics);
}

talp_gpu_status talp_gpu_plan_info(talp_gpu_plan* p, talp_gpu_plan_stats* out) {
    if (!p || !out) return fail(TALP_GPU_EINVAL, "null argument");
    out->n_metrics = p->n_metrics;
    out->records = p->L.n_records;
    out->segments = p->L.n_segs;
    out->kernels_per_launch = static_cast<uint32_t>(p->launches_per_run);
    out->sweep_items = kSweepShapes[p->L.shape].items;
    out->sweep_warps = kSweepShapes[p->L.shape].warps;
    out->sweep_stages = kSweepShapes[p->L.shape].stages;
    out->tiles_per_warp = static_cast<uint32_t>(p->L.tpw);
    out->sweep_grid = static_cast<uint32_t>(p->L.grid);
    out->slices_per_warp = static_cast<uint32_t>(p->L.spw);
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_plan_destroy(talp_gpu_plan* p) {
    if (!p) return TALP_GPU_OK;
    cudaSetDevice(p->c->device);
    cudaDeviceSynchronize();
    plan_release(p);
    return TALP_GPU_OK;
}

}  // extern "C"
