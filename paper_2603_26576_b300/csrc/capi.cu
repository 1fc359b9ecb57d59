// Host engine behind the C ABI: trace table, HBM admission, host-pointer
// staging, segment tables, launch sequence (prep -> sweep -> fix-up) and
// the result calls (finalize -> copy back).
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/talp_gpu.h"
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

#define TALP_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Per-trace device state: partial sums, windows, running carries, metrics.
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
    MetricsOut* metrics = nullptr; // [R]
    int cur = 0;
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
    b += align_up(sizeof(MetricsOut) * R, 256);
    return b;
}

// grow-only device buffer
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct PinBuf {
    void* p = nullptr;
    size_t cap = 0;
};

}  // namespace

void talp::set_last_error(const std::string& msg) { g_last_error = msg; }

struct talp_gpu_ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;
    size_t held = 0;
    std::unordered_map<uint64_t, TraceState*> traces;
    DevBuf ws;          // segment table, starts, fill jobs, payload, warp records, flags
    DevBuf stage;       // host-pointer record staging
    DevBuf sortbuf;     // ping-pong copies of the device segments being sorted
    PinBuf up, down;    // pinned upload / download scratch
    cudaEvent_t ev_up = nullptr;      // upload scratch free again
    cudaEvent_t ev_ws = nullptr;      // workspace/staging free again
    bool ws_used = false;
    int shape = kDefaultSweepShape;
    int min_tiles_per_warp = 4;
    // profiling
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    std::vector<uint64_t> ev_records;
    uint64_t kernel_launches = 0;
    int64_t wait_limit = 4000000000LL;   // cycles (~2 s at 2 GHz)
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

talp_gpu_status grow(talp_gpu_ctx* c, DevBuf& b, size_t need) {
    if (b.cap >= need) return TALP_GPU_OK;
    size_t cap = align_up(need + need / 4, 1 << 20);
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
    t->metrics = reinterpret_cast<MetricsOut*>(take(sizeof(MetricsOut) * R));
    *out = t;
    return TALP_GPU_OK;
}

// Host-side checks of one batch header (the records themselves are checked
// on the GPU).
talp_gpu_status check_batch(talp_gpu_ctx* c, const talp_gpu_trace_batch& b, uint64_t* n_host, uint64_t* n_dev,
                            uint32_t* m_out) {
    if (b.n_ranks == 0) return fail(TALP_GPU_EINVAL, "n_ranks must be >= 1");
    if (b.n_regions == 0 || b.n_regions > TALP_GPU_MAX_REGIONS)
        return fail(TALP_GPU_EINVAL, "n_regions must be in 1..8");
    if (b.reserved != 0) return fail(TALP_GPU_EINVAL, "reserved must be 0");
    if (b.flags & ~(TALP_GPU_DEVICE_PTRS | TALP_GPU_SORTED_BY_START | TALP_GPU_APPEND))
        return fail(TALP_GPU_EINVAL, "unknown flag bits");
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
    (void)c;
    return TALP_GPU_OK;
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
    cudaEventCreateWithFlags(&c->ev_ws, cudaEventDisableTiming);
    if (const char* s = getenv("TALP_GPU_SWEEP_SHAPE")) c->shape = atoi(s) % kNumSweepShapes;
    if (const char* s = getenv("TALP_GPU_TILES_PER_WARP")) c->min_tiles_per_warp = atoi(s) > 0 ? atoi(s) : 4;
    *out = c;
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_destroy(talp_gpu_ctx* c) {
    if (!c) return TALP_GPU_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto& kv : c->traces) free_trace(c, kv.second);
    c->traces.clear();
    dev_free(c, c->ws.p, c->ws.cap);
    dev_free(c, c->stage.p, c->stage.cap);
    dev_free(c, c->sortbuf.p, c->sortbuf.cap);
    if (c->up.p) cudaFreeHost(c->up.p);
    if (c->down.p) cudaFreeHost(c->down.p);
    if (c->ev_up) cudaEventDestroy(c->ev_up);
    if (c->ev_ws) cudaEventDestroy(c->ev_ws);
    for (auto& pr : c->ev_pending) {
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

    // ---- host-side validation and admission (nothing changes on failure)
    std::vector<uint64_t> nh(nb), nd(nb);
    std::vector<uint32_t> mm(nb);
    std::unordered_set<uint64_t> seen;
    size_t new_bytes = 0, stage_bytes = 0;
    uint64_t n_segs = 0, n_records = 0;
    uint32_t rmax = 1;
    for (size_t k = 0; k < nb; ++k) {
        const talp_gpu_trace_batch& b = batches[k];
        talp_gpu_status st = check_batch(c, b, &nh[k], &nd[k], &mm[k]);
        if (st != TALP_GPU_OK) return st;
        if (!seen.insert(b.trace_id).second) return fail(TALP_GPU_EINVAL, "trace id repeated in one call");
        auto it = c->traces.find(b.trace_id);
        if (b.flags & TALP_GPU_APPEND) {
            if (it == c->traces.end()) return fail(TALP_GPU_ENOTFOUND, "APPEND to an unknown trace");
            TraceState* t = it->second;
            if (t->n != b.n_ranks || t->R != b.n_regions ||
                memcmp(t->dpr.data(), b.devices_per_rank, sizeof(uint32_t) * b.n_ranks) != 0)
                return fail(TALP_GPU_EINVAL, "APPEND with a different trace shape");
        } else {
            bool reuse = it != c->traces.end() && it->second->n == b.n_ranks && it->second->R == b.n_regions &&
                         memcmp(it->second->dpr.data(), b.devices_per_rank, sizeof(uint32_t) * b.n_ranks) == 0;
            if (!reuse) {
                new_bytes += trace_bytes(b.n_ranks, mm[k], b.n_regions);
                if (it != c->traces.end()) new_bytes -= std::min(new_bytes, it->second->dbytes);
            }
        }
        if (!(b.flags & TALP_GPU_DEVICE_PTRS)) stage_bytes += nh[k] * 16 + nd[k] * 16 + align_up(nh[k], 16) + align_up(nd[k], 16) + 64;
        n_segs += mm[k] + b.n_ranks;
        n_records += nh[k] + nd[k];
        rmax = std::max(rmax, b.n_regions);
    }
    if (n_segs > 0xFFFFFFF0ull) return fail(TALP_GPU_EINVAL, "too many segments in one call");

    // sort stage sizes: device segments of batches that do not assert start order
    uint64_t sort_slots = 0, sort_recs = 0, sort_tiles = 0, n_dev_segs = 0;
    size_t n_backup_words = 0;
    for (size_t k = 0; k < nb; ++k) {
        const talp_gpu_trace_batch& b = batches[k];
        n_dev_segs += mm[k];
        if (b.flags & TALP_GPU_SORTED_BY_START) continue;
        sort_slots += mm[k];
        sort_recs += nd[k];
        for (uint32_t g = 0; g < mm[k]; ++g)
            sort_tiles += (b.dev_off[g + 1] - b.dev_off[g] + sort_tile_records() - 1) / sort_tile_records();
        if ((b.flags & TALP_GPU_APPEND) && mm[k]) n_backup_words += 3ull * b.n_regions * mm[k];
    }
    const bool sorting = sort_slots > 0;
    const size_t sortbuf_bytes = sorting ? 2 * (align_up(16 * sort_recs, 256) + align_up(sort_recs + 64, 256)) : 0;

    // workspace layout (device): [segs][seg_start][fill jobs][payload][wrec][seg_flags][gstatus]
    const int shape = c->shape;
    const int tile = sweep_tile(shape);
    const int warps = kSweepShapes[shape].warps;
    int cps = sweep_ctas_per_sm(shape, static_cast<int>(rmax));
    if (cps <= 0) return fail(TALP_GPU_ECUDA, "sweep kernel cannot be resident");
    const uint64_t tiles = (n_records + tile - 1) / tile;
    uint64_t want_warps = (tiles + c->min_tiles_per_warp - 1) / c->min_tiles_per_warp;
    const uint64_t max_warps = static_cast<uint64_t>(c->num_sms) * cps * warps;
    if (want_warps > max_warps) want_warps = max_warps;
    if (want_warps < 1) want_warps = 1;
    const int grid = static_cast<int>((want_warps + warps - 1) / warps);
    const int full_grid = static_cast<int>(max_warps / warps);   // re-sweep: size unknown on the host
    const uint32_t n_wrec = static_cast<uint32_t>(grid) * warps;
    const uint32_t n_wrec_cap = static_cast<uint32_t>(sorting ? std::max(grid, full_grid) : grid) * warps;

    // payload per trace: hwin [n][R][2], dev_rank [m] (only at creation), TraceDev
    size_t payload_words = 0;
    for (size_t k = 0; k < nb; ++k)
        payload_words += 2ull * batches[k].n_ranks * batches[k].n_regions + mm[k] + sizeof(TraceDev) / 8;
    const size_t n_jobs_max = 8 * nb + 2;   // <= 8 per trace + seg flags + status
    size_t off_segs = 0;
    size_t off_start = align_up(off_segs + sizeof(SegDesc) * n_segs, 256);
    size_t off_jobs = align_up(off_start + sizeof(uint64_t) * (n_segs + 1), 256);
    size_t off_rest = align_up(off_jobs + sizeof(FillJob) * n_jobs_max, 256);
    size_t off_sctl = align_up(off_rest + sizeof(int64_t*) * (sorting ? n_segs : 0), 256);
    size_t off_pay = align_up(off_sctl + sizeof(SortCtl), 256);
    size_t up_bytes = align_up(off_pay + 8 * payload_words, 256);
    // device-only part
    size_t off_wrec = up_bytes;
    size_t off_flags = align_up(off_wrec + sizeof(WarpRec) * n_wrec_cap, 256);
    size_t off_gst = align_up(off_flags + sizeof(uint32_t) * (n_segs + 1), 256);
    size_t off_bk = align_up(off_gst + 256, 256);
    size_t off_slist = align_up(off_bk + 8 * n_backup_words, 256);
    size_t off_srb = align_up(off_slist + 4 * sort_slots, 256);
    size_t off_stb = align_up(off_srb + 8 * sort_slots, 256);
    size_t off_smn = align_up(off_stb + 8 * (sort_slots + 1), 256);
    size_t off_smx = align_up(off_smn + 8 * sort_slots, 256);
    size_t off_hist = align_up(off_smx + 8 * sort_slots, 256);
    size_t off_offs = align_up(off_hist + 4 * 256 * sort_tiles, 256);
    size_t off_rsegs = align_up(off_offs + 8 * 256 * sort_tiles, 256);
    size_t off_rstart = align_up(off_rsegs + sizeof(SegDesc) * (sorting ? n_dev_segs : 0), 256);
    size_t ws_bytes = align_up(off_rstart + 8 * (sorting ? n_dev_segs + 1 : 0), 256);

    size_t extra = new_bytes;
    if (c->ws.cap < ws_bytes) extra += align_up(ws_bytes + ws_bytes / 4, 1 << 20) - c->ws.cap;
    if (c->stage.cap < stage_bytes) extra += align_up(stage_bytes + stage_bytes / 4, 1 << 20) - c->stage.cap;
    if (c->sortbuf.cap < sortbuf_bytes)
        extra += align_up(sortbuf_bytes + sortbuf_bytes / 4, 1 << 20) - c->sortbuf.cap;
    if (c->held + extra > c->budget)
        return fail(TALP_GPU_ENOMEM, "admission: the ingest needs " + std::to_string(extra) +
                                         " more device bytes than the budget leaves");

    // previous ingest must be done with the workspace/staging before reuse
    if (c->ws_used) TALP_CUDA(cudaStreamWaitEvent(stream, c->ev_ws, 0));
    talp_gpu_status st = grow(c, c->ws, ws_bytes);
    if (st != TALP_GPU_OK) return st;
    if (stage_bytes) {
        st = grow(c, c->stage, stage_bytes);
        if (st != TALP_GPU_OK) return st;
    }
    if (sortbuf_bytes) {
        st = grow(c, c->sortbuf, sortbuf_bytes);
        if (st != TALP_GPU_OK) return st;
    }
    TALP_CUDA(cudaEventSynchronize(c->ev_up));   // upload scratch no longer read by a pending copy
    st = grow_pinned(c->up, up_bytes);
    if (st != TALP_GPU_OK) return st;

    // ---- trace states
    std::vector<TraceState*> ts(nb);
    for (size_t k = 0; k < nb; ++k) {
        const talp_gpu_trace_batch& b = batches[k];
        auto it = c->traces.find(b.trace_id);
        if (it != c->traces.end() && it->second->n == b.n_ranks && it->second->R == b.n_regions &&
            memcmp(it->second->dpr.data(), b.devices_per_rank, sizeof(uint32_t) * b.n_ranks) == 0) {
            ts[k] = it->second;
            continue;
        }
        if (it != c->traces.end()) {
            cudaStreamSynchronize(stream);
            free_trace(c, it->second);
            c->traces.erase(it);
        }
        TraceState* t = nullptr;
        st = alloc_trace(c, b.trace_id, b.n_ranks, b.devices_per_rank, b.n_regions, &t);
        if (st != TALP_GPU_OK) return st;
        c->traces[b.trace_id] = t;
        ts[k] = t;
    }

    // ---- host-pointer records: copy into staging
    char* up = static_cast<char*>(c->up.p);
    char* wsd = static_cast<char*>(c->ws.p);
    std::vector<const int64_t*> hse(nb), dse(nb);
    std::vector<const uint8_t*> hst(nb), dtg(nb), hst_end(nb), dtg_end(nb);
    size_t so = 0;
    char* stg = static_cast<char*>(c->stage.p);
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
            char* a = put(b.host_se, nh[k] * 16);
            char* bb = put(b.dev_se, nd[k] * 16);
            char* cc = put(b.host_state, nh[k]);
            char* dd = put(b.dev_tag, nd[k]);
            if (!a || !bb || !cc || !dd) return cuda_fail(cudaGetLastError(), "cudaMemcpyAsync (records)");
            hse[k] = reinterpret_cast<const int64_t*>(a);
            dse[k] = reinterpret_cast<const int64_t*>(bb);
            hst[k] = reinterpret_cast<const uint8_t*>(cc);
            dtg[k] = reinterpret_cast<const uint8_t*>(dd);
        }
        auto floor16 = [](const uint8_t* p) {
            return reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(p) & ~static_cast<uintptr_t>(15));
        };
        hst_end[k] = floor16(hst[k] + nh[k]);
        dtg_end[k] = floor16(dtg[k] + nd[k]);
    }

    // ---- segment table, fill jobs, payload (one upload)
    SegDesc* sd = reinterpret_cast<SegDesc*>(up + off_segs);
    uint64_t* sstart = reinterpret_cast<uint64_t*>(up + off_start);
    FillJob* jobs = reinterpret_cast<FillJob*>(up + off_jobs);
    int64_t* pay = reinterpret_cast<int64_t*>(up + off_pay);
    int64_t* pay_dev = reinterpret_cast<int64_t*>(wsd + off_pay);
    uint32_t* seg_flags = reinterpret_cast<uint32_t*>(wsd + off_flags);
    uint32_t* gstatus = reinterpret_cast<uint32_t*>(wsd + off_gst);
    const int64_t** restore = reinterpret_cast<const int64_t**>(up + off_rest);
    size_t pw = 0, bk_used = 0;
    uint32_t nj = 0;
    uint64_t si = 0, pos = 0;
    for (size_t k = 0; k < nb; ++k) {
        const talp_gpu_trace_batch& b = batches[k];
        TraceState* t = ts[k];
        const bool append = (b.flags & TALP_GPU_APPEND) != 0;
        const uint32_t n = t->n, m = t->m, R = t->R;
        int64_t* bkd = nullptr;   // pre-ingest device sums (APPEND + sorting)
        int64_t* cin = t->carry[t->cur];
        int64_t* cout = t->carry[t->cur ^ 1];
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
                bkd = reinterpret_cast<int64_t*>(wsd + off_bk) + bk_used;
                bk_used += 3ull * R * m;
                jobs[nj++] = FillJob{bkd, 3ull * m * R, 0, t->dsum};
            }
        }
        const uint8_t seg_flags0 = (b.flags & TALP_GPU_SORTED_BY_START) ? 0 : kSegSortable;
        // device segments, then host segments
        for (uint32_t g = 0; g < m; ++g) {
            SegDesc& s = sd[si];
            const uint64_t o = b.dev_off[g];
            s.se = dse[k] + 2 * o;
            s.tag = dtg[k] + o;
            s.tag_limit = dtg_end[k];
            s.sums = t->dsum + static_cast<size_t>(g) * R * 3;
            uint32_t rank = static_cast<uint32_t>(dr[g]);
            s.win = t->hwin + static_cast<size_t>(rank) * R * 2;
            s.status = t->status;
            s.carry_in = cin + 3ull * g;
            s.carry_out = cout + 3ull * g;
            s.n = b.dev_off[g + 1] - o;
            s.R = static_cast<uint16_t>(R);
            s.is_host = 0;
            memset(s.pad, 0, sizeof(s.pad));
            s.pad[0] = seg_flags0;
            if (sorting) restore[si] = bkd ? bkd + static_cast<size_t>(g) * R * 3 : nullptr;
            sstart[si] = pos;
            pos += s.n;
            ++si;
        }
        for (uint32_t i = 0; i < n; ++i) {
            SegDesc& s = sd[si];
            const uint64_t o = b.host_off[i];
            s.se = hse[k] + 2 * o;
            s.tag = hst[k] + o;
            s.tag_limit = hst_end[k];
            s.sums = t->hsum + static_cast<size_t>(i) * R * 3;
            s.win = t->hwin + static_cast<size_t>(i) * R * 2;
            s.status = t->status;
            s.carry_in = nullptr;
            s.carry_out = nullptr;
            s.n = b.host_off[i + 1] - o;
            s.R = static_cast<uint16_t>(R);
            s.is_host = 1;
            memset(s.pad, 0, sizeof(s.pad));
            sstart[si] = pos;
            pos += s.n;
            ++si;
        }
    }
    sstart[si] = pos;
    jobs[nj++] = FillJob{reinterpret_cast<int64_t*>(seg_flags), (n_segs + 2) / 2, 0, nullptr};
    jobs[nj++] = FillJob{reinterpret_cast<int64_t*>(gstatus), 1, 0, nullptr};
    if (nj > n_jobs_max || pw > payload_words || si != n_segs || bk_used > n_backup_words)
        return fail(TALP_GPU_ECUDA, "internal: upload table overflow");
    if (sorting) {
        SortCtl sc{};
        sc.list = reinterpret_cast<uint32_t*>(wsd + off_slist);
        sc.rec_base = reinterpret_cast<uint64_t*>(wsd + off_srb);
        sc.tile_base = reinterpret_cast<uint64_t*>(wsd + off_stb);
        sc.mn = reinterpret_cast<int64_t*>(wsd + off_smn);
        sc.mx = reinterpret_cast<int64_t*>(wsd + off_smx);
        sc.hist = reinterpret_cast<uint32_t*>(wsd + off_hist);
        sc.offs = reinterpret_cast<uint64_t*>(wsd + off_offs);
        char* sb = static_cast<char*>(c->sortbuf.p);
        const size_t se_b = align_up(16 * sort_recs, 256), tg_b = align_up(sort_recs + 64, 256);
        for (int q = 0; q < 2; ++q) {
            char* base = sb + q * (se_b + tg_b);
            sc.buf_se[q] = reinterpret_cast<int64_t*>(base);
            sc.buf_tag[q] = reinterpret_cast<uint8_t*>(base + se_b);
            sc.buf_tag_limit[q] = reinterpret_cast<const uint8_t*>(
                reinterpret_cast<uintptr_t>(base + se_b + tg_b) & ~static_cast<uintptr_t>(15));
        }
        sc.restore = reinterpret_cast<const int64_t* const*>(wsd + off_rest);
        memcpy(up + off_sctl, &sc, sizeof(SortCtl));
    }

    TALP_CUDA(cudaMemcpyAsync(wsd, up, up_bytes, cudaMemcpyHostToDevice, stream));
    TALP_CUDA(cudaEventRecord(c->ev_up, stream));

    // ---- launches
    TALP_CUDA(launch_prep(reinterpret_cast<const FillJob*>(wsd + off_jobs), nj, stream));
    ++c->kernel_launches;
    const SegDesc* dsegs = reinterpret_cast<const SegDesc*>(wsd + off_segs);
    const uint64_t* dstart = reinterpret_cast<const uint64_t*>(wsd + off_start);
    WarpRec* wrec = reinterpret_cast<WarpRec*>(wsd + off_wrec);
    if (n_records > 0) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (c->profiling) {
            e0 = take_event(c);
            e1 = take_event(c);
            TALP_CUDA(cudaEventRecord(e0, stream));
        }
        TALP_CUDA(launch_sweep(shape, static_cast<int>(rmax), grid, dsegs, dstart, static_cast<uint32_t>(n_segs), wrec,
                               seg_flags, gstatus, c->wait_limit, stream));
        if (c->profiling) {
            TALP_CUDA(cudaEventRecord(e1, stream));
            c->ev_pending.emplace_back(e0, e1);
            c->ev_records.push_back(n_records);
        }
        TALP_CUDA(launch_fixup(dsegs, dstart, wrec, n_wrec, seg_flags, stream));
        c->kernel_launches += 2;
        if (sorting) {
            // a2: sort the device segments found out of order, re-sweep them
            SortCtl* sctl = reinterpret_cast<SortCtl*>(wsd + off_sctl);
            SegDesc* rsegs = reinterpret_cast<SegDesc*>(wsd + off_rsegs);
            uint64_t* rstart = reinterpret_cast<uint64_t*>(wsd + off_rstart);
            const uint64_t gt = std::min<uint64_t>(sort_tiles, static_cast<uint64_t>(c->num_sms) * 8);
            const uint64_t gs = std::min<uint64_t>(sort_slots, static_cast<uint64_t>(c->num_sms) * 4);
            TALP_CUDA(launch_sort_stage(dsegs, static_cast<uint32_t>(n_segs), static_cast<uint32_t>(n_dev_segs),
                                        seg_flags, sctl, rsegs, rstart, static_cast<int>(std::max<uint64_t>(gt, 1)),
                                        static_cast<int>(std::max<uint64_t>(gs, 1)), stream));
            TALP_CUDA(launch_sweep(shape, static_cast<int>(rmax), full_grid, rsegs, rstart,
                                   static_cast<uint32_t>(n_dev_segs), wrec, seg_flags, gstatus, c->wait_limit, stream));
            TALP_CUDA(launch_fixup(rsegs, rstart, wrec, static_cast<uint32_t>(full_grid) * warps, seg_flags, stream));
            c->kernel_launches += 2 + 24 + 1 + 2;
        }
    }
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
    std::vector<TraceState*> ts;
    for (size_t k = 0; k < n; ++k) {
        auto it = c->traces.find(ids[k]);
        if (it == c->traces.end()) return fail(TALP_GPU_ENOTFOUND, "unknown trace id " + std::to_string(ids[k]));
        TraceState* t = it->second;
        if (region == TALP_GPU_ALL_REGIONS) {
            if (n != 1) return fail(TALP_GPU_EINVAL, "TALP_GPU_ALL_REGIONS takes one trace");
            for (uint32_t r = 0; r < t->R; ++r) {
                jobs.push_back(FinalizeJob{t->tdev, out_dev_user ? out_dev_user + r : t->metrics + r, r, 0});
                ts.push_back(t);
            }
        } else {
            if (region >= t->R) return fail(TALP_GPU_EINVAL, "region out of range");
            jobs.push_back(FinalizeJob{t->tdev, out_dev_user ? out_dev_user + k : t->metrics + region, region, 0});
            ts.push_back(t);
        }
    }
    const size_t jb = sizeof(FinalizeJob) * jobs.size();
    TALP_CUDA(cudaEventSynchronize(c->ev_up));
    talp_gpu_status st = grow_pinned(c->up, jb);
    if (st != TALP_GPU_OK) return st;
    if (c->ws_used) TALP_CUDA(cudaStreamWaitEvent(stream, c->ev_ws, 0));
    st = grow(c, c->ws, jb + 256);
    if (st != TALP_GPU_OK) return st;
    memcpy(c->up.p, jobs.data(), jb);
    TALP_CUDA(cudaMemcpyAsync(c->ws.p, c->up.p, jb, cudaMemcpyHostToDevice, stream));
    TALP_CUDA(cudaEventRecord(c->ev_up, stream));
    TALP_CUDA(launch_finalize(static_cast<const FinalizeJob*>(c->ws.p), static_cast<uint32_t>(jobs.size()), stream));
    ++c->kernel_launches;
    TALP_CUDA(cudaEventRecord(c->ev_ws, stream));
    c->ws_used = true;
    if (!sync) return TALP_GPU_OK;
    st = grow_pinned(c->down, sizeof(MetricsOut) * jobs.size());
    if (st != TALP_GPU_OK) return st;
    MetricsOut* dn = static_cast<MetricsOut*>(c->down.p);
    for (size_t k = 0; k < jobs.size(); ++k)
        TALP_CUDA(cudaMemcpyAsync(dn + k, jobs[k].out, sizeof(MetricsOut), cudaMemcpyDeviceToHost, stream));
    TALP_CUDA(cudaStreamSynchronize(stream));
    memcpy(out_host, dn, sizeof(MetricsOut) * jobs.size());
    talp_gpu_status res = TALP_GPU_OK;
    for (size_t k = 0; k < jobs.size(); ++k) {
        const uint32_t f = out_host[k].flags;
        if (f & TALP_GPU_M_TIMEOUT) {
            if (res == TALP_GPU_OK) res = fail(TALP_GPU_ETIMEDOUT, "a device-side wait ran out during ingest");
        } else if (f & (TALP_GPU_M_INVALID | TALP_GPU_M_UNSORTED)) {
            if (res == TALP_GPU_OK)
                res = fail(TALP_GPU_EINVAL, (f & TALP_GPU_M_INVALID) ? "invalid record (end < start or bad kind/state)"
                                                                     : "device records out of start order");
        }
    }
    return res;
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
        for (auto& kv : c->traces) free_trace(c, kv.second);
        c->traces.clear();
        return TALP_GPU_OK;
    }
    auto it = c->traces.find(trace_id);
    if (it == c->traces.end()) return fail(TALP_GPU_ENOTFOUND, "unknown trace id");
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
    out->kernel_launches = c->kernel_launches;
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_memory(talp_gpu_ctx* c, size_t* held, size_t* budget) {
    if (!c) return fail(TALP_GPU_EINVAL, "null context");
    if (held) *held = c->held;
    if (budget) *budget = c->budget;
    return TALP_GPU_OK;
}

}  // extern "C"
