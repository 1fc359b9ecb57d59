// Serving loop: at-runtime monitoring of many jobs with continuous batching
// (the metrics are available while the application runs, Sec. 3.2).
//
// Threads:
//  - clients (any number) call submit / query / open / close / drain;
//  - the server thread owns the context.  It admits jobs, forms fold waves
//    (one APPEND ingest holding the next pending slice of every job that has
//    one; at most kMaxWavesInFlight waves are queued on the GPU, so slices
//    that arrive meanwhile gather into the next, larger wave), batches every
//    ready query into one finalize launch on a high-priority stream, and
//    retires completed waves;
//  - the completion thread waits for each query batch, copies the answers
//    out and wakes the clients.
// The running state of every job (per-rank and per-device sums and chain
// carries of Sec. 4.1/4.2) stays on the device in the context's trace table.
//
// Consistency: a query launch waits for the last wave holding a slice of
// its job, and every wave enqueued after a query launch waits for that
// launch's finalize kernel, so a finalize never reads state that a fold is
// changing.  A query is issued once every slice its job had when the query
// arrived sits in an enqueued wave.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/talp_gpu.h"
#include "engine.h"
#include "kernels.h"

using namespace talp;

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kMaxWavesInFlight = 2;
constexpr uint32_t kMaxUnitsPerJob = 64 * 1024;   // ranks, and devices, of one job
constexpr size_t kQuerySlots = 4;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Slice {
    int chunk = -1;
    uint32_t flags = 0;
    bool raw = false;              // raw activity records (raw_dev / raw_off below), folded by the raw adapter
    const uint8_t* raw_dev = nullptr;
    const int64_t* host_se = nullptr;
    const uint8_t* host_state = nullptr;
    const uint64_t* host_off = nullptr;
    const int64_t* dev_se = nullptr;
    const uint8_t* dev_tag = nullptr;
    const uint64_t* dev_off = nullptr;
    uint64_t records = 0;
};

struct Job {
    uint64_t id = 0;
    uint32_t n = 0, m = 0, R = 0;
    std::vector<uint32_t> dpr;
    std::vector<int64_t> win;      // [R][n][2]
    std::vector<uint32_t> smask;   // [n][8] declared streams: the union of every raw submission's masks
    std::deque<Slice> pending;
    uint64_t submitted = 0;        // slices accepted
    uint64_t enqueued = 0;         // slices in enqueued waves
    int64_t last_wave = -1;        // latest wave that touched the job's state
    talp_gpu_status error = TALP_GPU_OK;
};

struct Query {
    uint64_t job = 0;
    uint32_t region = 0;
    uint32_t n_out = 0;
    uint64_t need = 0;             // slices that must be enqueued first
    talp_gpu_metrics* out = nullptr;
    // a thread-tree query instead (tout set): the client's process table,
    // valid while it waits
    talp_gpu_thread_tree* tout = nullptr;
    const uint32_t* proc_off = nullptr;
    uint32_t n_procs = 0;
    talp_gpu_status st = TALP_GPU_OK;
    bool done = false;
    Clock::time_point t0;
};

enum CmdKind { CMD_OPEN, CMD_CLOSE };
struct Cmd {
    CmdKind kind;
    Job* job = nullptr;            // CMD_OPEN: the job to admit
    uint64_t id = 0;               // CMD_CLOSE
    talp_gpu_status st = TALP_GPU_OK;
    std::string msg;
    bool done = false;
};

struct Wave {
    int64_t id = 0;
    cudaEvent_t ev = nullptr;
    std::vector<int> chunks;
    uint64_t records = 0, slices = 0;
    bool fold = true;              // false: the admission ingest of a job
};

struct QSlot {
    FinalizeJob* d_jobs = nullptr;
    MetricsOut* d_out = nullptr;
    FinalizeJob* h_jobs = nullptr;
    MetricsOut* h_out = nullptr;
    // thread-tree queries: jobs and results, and their process tables
    ThreadJob* d_tjobs = nullptr;
    ThreadOut* d_tout = nullptr;
    ThreadJob* h_tjobs = nullptr;
    ThreadOut* h_tout = nullptr;
    uint32_t* d_po = nullptr;
    uint32_t* h_po = nullptr;
    size_t po_cap = 0;             // entries of d_po / h_po
    cudaEvent_t ev_fin = nullptr;  // finalize kernel done
    cudaEvent_t ev = nullptr;      // answers on the host side
    std::vector<Query*> qs;
    bool busy = false;             // guarded by the server mutex
};

}  // namespace

struct talp_gpu_server {
    talp_gpu_ctx* ctx = nullptr;
    talp_gpu_server_config cfg{};
    int device = 0;
    cudaStream_t s_fold = nullptr, s_query = nullptr;
    size_t chunk_bytes = 0;
    std::vector<char*> chunks;
    std::vector<QSlot> qslots;
    size_t qslot_entries = 0;

    std::mutex mu;
    std::condition_variable cv_work;   // wakes the server thread (work_gen changed)
    std::condition_variable cv_done;   // wakes clients (commands, queries, drain)
    std::condition_variable cv_chunk;  // wakes submitters waiting for staging
    uint64_t work_gen = 0;
    std::unordered_map<uint64_t, Job*> jobs;
    std::vector<int> free_chunks;
    std::deque<Query*> queries;
    std::deque<Cmd*> cmds;
    bool stop = false;

    // server-thread only
    std::deque<Wave> inflight;
    std::vector<cudaEvent_t> ev_pool;
    int64_t next_wave = 0;
    cudaEvent_t fin_to_wait = nullptr;  // finalize launch the next wave must follow

    // server -> completion thread
    std::mutex qmu;
    std::condition_variable qcv;
    std::deque<int> qinflight;
    bool stop_done = false;

    std::thread th_serve, th_done;
    bool held = false;                 // counted as a user of the context

    // statistics (under mu)
    uint64_t slices_submitted = 0, slices_folded = 0, records_folded = 0, waves = 0, queries_answered = 0,
             query_batches = 0;
    uint64_t unfinished_waves = 0;
    std::vector<double> lat_ms;
};

namespace {

void wake(talp_gpu_server* s) {
    ++s->work_gen;
    s->cv_work.notify_one();
}

template <typename T>
talp_gpu_status check_flags(const T* out, uint32_t n) {
    for (uint32_t k = 0; k < n; ++k) {
        if (out[k].flags & TALP_GPU_M_TIMEOUT) return TALP_GPU_ETIMEDOUT;
        if (out[k].flags & (TALP_GPU_M_INVALID | TALP_GPU_M_UNSORTED)) return TALP_GPU_EINVAL;
    }
    return TALP_GPU_OK;
}

// Room for `need` process-table entries in a free query slot (server thread).
bool grow_po(QSlot& q, size_t need) {
    if (need <= q.po_cap) return true;
    size_t cap = q.po_cap ? q.po_cap : 4096;
    while (cap < need) cap *= 2;
    if (q.d_po) cudaFree(q.d_po);
    if (q.h_po) cudaFreeHost(q.h_po);
    q.d_po = nullptr;
    q.h_po = nullptr;
    q.po_cap = 0;
    if (cudaMalloc(&q.d_po, sizeof(uint32_t) * cap) != cudaSuccess) return false;
    if (cudaMallocHost(&q.h_po, sizeof(uint32_t) * cap) != cudaSuccess) return false;
    q.po_cap = cap;
    return true;
}

cudaEvent_t take_event(talp_gpu_server* s) {
    if (!s->ev_pool.empty()) {
        cudaEvent_t e = s->ev_pool.back();
        s->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

// Mark the end of a wave's launches on the fold stream.
void record_wave(talp_gpu_server* s, Wave& w) {
    w.ev = take_event(s);
    cudaEventRecord(w.ev, s->s_fold);
}

// Admission (lock held on entry and exit): slot check, then an empty ingest
// creates the job's device state; the context refuses it with ENOMEM past
// its HBM budget.
talp_gpu_status admit(talp_gpu_server* s, Job* j, std::unique_lock<std::mutex>& lk, std::string& msg) {
    if (s->jobs.size() >= s->cfg.max_jobs) {
        msg = "server: all job slots are taken";
        return TALP_GPU_EBUSY;
    }
    if (s->jobs.count(j->id)) {
        msg = "server: job id already open";
        return TALP_GPU_EINVAL;
    }
    std::vector<uint64_t> hoff(j->n + 1, 0), doff(j->m + 1, 0);
    talp_gpu_trace_batch b{};
    b.trace_id = j->id;
    b.n_ranks = j->n;
    b.n_regions = j->R;
    b.flags = TALP_GPU_SORTED_BY_START;
    b.devices_per_rank = j->dpr.data();
    b.region_window = j->win.data();
    b.host_off = hoff.data();
    b.dev_off = doff.data();
    lk.unlock();
    if (s->fin_to_wait) cudaStreamWaitEvent(s->s_fold, s->fin_to_wait, 0);
    s->fin_to_wait = nullptr;
    talp_gpu_status st = talp_gpu_ingest_events(s->ctx, &b, 1, s->s_fold);
    if (st != TALP_GPU_OK) msg = talp_gpu_last_error();
    Wave w;
    w.fold = false;
    if (st == TALP_GPU_OK) record_wave(s, w);
    lk.lock();
    if (st != TALP_GPU_OK) return st;
    w.id = s->next_wave++;
    j->last_wave = w.id;
    s->inflight.push_back(w);
    ++s->unfinished_waves;
    s->jobs[j->id] = j;
    return TALP_GPU_OK;
}

void close_job_locked(talp_gpu_server* s, Cmd* c, std::unique_lock<std::mutex>& lk) {
    auto it = s->jobs.find(c->id);
    if (it == s->jobs.end()) {
        c->st = TALP_GPU_ENOTFOUND;
        c->msg = "server: unknown job";
        return;
    }
    Job* j = it->second;
    s->jobs.erase(it);
    for (Slice& sl : j->pending) s->free_chunks.push_back(sl.chunk);
    s->cv_chunk.notify_all();
    // queued queries of the job end with ENOTFOUND
    for (auto qi = s->queries.begin(); qi != s->queries.end();) {
        if ((*qi)->job == c->id) {
            (*qi)->st = TALP_GPU_ENOTFOUND;
            (*qi)->done = true;
            qi = s->queries.erase(qi);
        } else {
            ++qi;
        }
    }
    lk.unlock();
    cudaStreamSynchronize(s->s_fold);
    cudaStreamSynchronize(s->s_query);
    c->st = talp_gpu_reset(s->ctx, j->id);
    if (c->st != TALP_GPU_OK) c->msg = talp_gpu_last_error();
    lk.lock();
    delete j;
}

// Fold waves: the next pending slice of every job, while the GPU queue has room.
void form_waves(talp_gpu_server* s, std::unique_lock<std::mutex>& lk) {
    while (s->inflight.size() < kMaxWavesInFlight) {
        std::vector<Slice> take;
        std::vector<Job*> owners;
        for (auto& kv : s->jobs) {
            Job* j = kv.second;
            if (j->pending.empty() || j->error != TALP_GPU_OK) continue;
            take.push_back(j->pending.front());
            owners.push_back(j);
            j->pending.pop_front();
            ++j->enqueued;
        }
        if (take.empty()) return;
        std::vector<talp_gpu_trace_batch> bs;
        std::vector<talp_gpu_raw_batch> rs;
        std::vector<std::vector<uint32_t>> masks;   // copied under the lock: submitters may replace them
        masks.reserve(take.size());
        for (size_t k = 0; k < take.size(); ++k) {
            const Job* j = owners[k];
            const Slice& sl = take[k];
            if (sl.raw) {
                talp_gpu_raw_batch r;
                memset(&r, 0, sizeof(r));
                r.trace_id = j->id;
                r.n_ranks = j->n;
                r.n_regions = j->R;
                r.flags = TALP_GPU_APPEND | (sl.flags & TALP_GPU_HOLD_BACK);
                r.devices_per_rank = j->dpr.data();
                r.region_window = j->win.data();
                r.host_se = sl.host_se;
                r.host_state = sl.host_state;
                r.host_off = sl.host_off;
                r.raw_se = sl.dev_se;
                r.raw_tag = sl.dev_tag;
                r.raw_dev = sl.raw_dev;
                r.raw_off = sl.dev_off;
                masks.push_back(j->smask);
                r.stream_mask = masks.back().data();
                rs.push_back(r);
                continue;
            }
            talp_gpu_trace_batch b;
            memset(&b, 0, sizeof(b));
            b.trace_id = j->id;
            b.n_ranks = j->n;
            b.n_regions = j->R;
            b.flags = TALP_GPU_APPEND | (sl.flags & TALP_GPU_SORTED_BY_START);
            b.devices_per_rank = j->dpr.data();
            b.region_window = j->win.data();
            b.host_se = sl.host_se;
            b.host_state = sl.host_state;
            b.host_off = sl.host_off;
            b.dev_se = sl.dev_se;
            b.dev_tag = sl.dev_tag;
            b.dev_off = sl.dev_off;
            bs.push_back(b);
        }
        lk.unlock();
        if (s->fin_to_wait) cudaStreamWaitEvent(s->s_fold, s->fin_to_wait, 0);
        s->fin_to_wait = nullptr;
        // plain slices in one ingest; raw ones in one call of the raw adapter
        // (hold-back state per job lives in the context, keyed by the job id)
        talp_gpu_status st = TALP_GPU_OK, st_raw = TALP_GPU_OK;
        if (!bs.empty()) st = talp_gpu_ingest_events(s->ctx, bs.data(), bs.size(), s->s_fold);
        if (!rs.empty()) st_raw = talp_gpu_ingest_raw(s->ctx, rs.data(), rs.size(), s->s_fold);
        Wave w;
        record_wave(s, w);
        lk.lock();
        w.id = s->next_wave++;
        for (size_t k = 0; k < take.size(); ++k) {
            owners[k]->last_wave = w.id;
            const talp_gpu_status sk = take[k].raw ? st_raw : st;
            if (sk != TALP_GPU_OK) owners[k]->error = sk;   // the job's state is no longer defined
            w.chunks.push_back(take[k].chunk);
            w.records += take[k].records;
        }
        w.slices = take.size();
        s->inflight.push_back(w);
        ++s->unfinished_waves;
        ++s->waves;
    }
}

// All ready queries in one finalize launch (lock held; released around CUDA calls).
void issue_queries(talp_gpu_server* s, std::unique_lock<std::mutex>& lk) {
    if (s->queries.empty()) return;
    int slot = -1;
    for (size_t k = 0; k < s->qslots.size(); ++k)
        if (!s->qslots[k].busy) {
            slot = static_cast<int>(k);
            break;
        }
    if (slot < 0) return;   // the completion thread frees one and wakes us
    QSlot& q = s->qslots[slot];
    q.qs.clear();
    int64_t need_wave = -1;
    size_t e = 0, et = 0, po_used = 0;
    size_t po_need = 0;
    for (const Query* r : s->queries)
        if (r->tout) po_need += r->n_procs + 1;
    if (po_need && !grow_po(q, po_need)) {
        // no room for any process table now: answer the thread queries with ENOMEM
        for (auto qi = s->queries.begin(); qi != s->queries.end();) {
            if ((*qi)->tout) {
                (*qi)->st = TALP_GPU_ENOMEM;
                (*qi)->done = true;
                qi = s->queries.erase(qi);
            } else {
                ++qi;
            }
        }
        s->cv_done.notify_all();
    }
    for (auto qi = s->queries.begin(); qi != s->queries.end();) {
        Query* r = *qi;
        auto it = s->jobs.find(r->job);
        if (it == s->jobs.end() || it->second->error != TALP_GPU_OK) {
            r->st = it == s->jobs.end() ? TALP_GPU_ENOTFOUND : it->second->error;
            r->done = true;
            qi = s->queries.erase(qi);
            s->cv_done.notify_all();
            continue;
        }
        Job* j = it->second;
        const bool thr = r->tout != nullptr;
        if (j->enqueued < r->need || (thr ? et : e) + r->n_out > s->qslot_entries ||
            (thr && po_used + r->n_procs + 1 > q.po_cap)) {
            ++qi;
            continue;
        }
        uint32_t R = 0;
        const TraceDev* td = trace_device_desc(s->ctx, j->id, &R);
        const uint32_t r0 = r->region == TALP_GPU_ALL_REGIONS ? 0 : r->region;
        if (thr) {
            memcpy(q.h_po + po_used, r->proc_off, sizeof(uint32_t) * (r->n_procs + 1));
            for (uint32_t k = 0; k < r->n_out; ++k, ++et)
                q.h_tjobs[et] = ThreadJob{td, q.d_tout + et, q.d_po + po_used, r->n_procs, r0 + k};
            po_used += r->n_procs + 1;
        } else {
            for (uint32_t k = 0; k < r->n_out; ++k, ++e) q.h_jobs[e] = FinalizeJob{td, q.d_out + e, r0 + k, 0};
        }
        need_wave = std::max(need_wave, j->last_wave);
        q.qs.push_back(r);
        qi = s->queries.erase(qi);
    }
    if (q.qs.empty()) return;
    q.busy = true;
    cudaEvent_t wait_ev = nullptr;
    for (const Wave& w : s->inflight)
        if (w.id == need_wave) wait_ev = w.ev;
    ++s->query_batches;
    lk.unlock();
    if (wait_ev) cudaStreamWaitEvent(s->s_query, wait_ev, 0);
    if (e) {
        cudaMemcpyAsync(q.d_jobs, q.h_jobs, sizeof(FinalizeJob) * e, cudaMemcpyHostToDevice, s->s_query);
        launch_finalize(q.d_jobs, static_cast<uint32_t>(e), s->s_query);
    }
    if (et) {
        cudaMemcpyAsync(q.d_po, q.h_po, sizeof(uint32_t) * po_used, cudaMemcpyHostToDevice, s->s_query);
        cudaMemcpyAsync(q.d_tjobs, q.h_tjobs, sizeof(ThreadJob) * et, cudaMemcpyHostToDevice, s->s_query);
        launch_thread_tree(q.d_tjobs, static_cast<uint32_t>(et), s->s_query);
    }
    cudaEventRecord(q.ev_fin, s->s_query);
    if (e) cudaMemcpyAsync(q.h_out, q.d_out, sizeof(MetricsOut) * e, cudaMemcpyDeviceToHost, s->s_query);
    if (et) cudaMemcpyAsync(q.h_tout, q.d_tout, sizeof(ThreadOut) * et, cudaMemcpyDeviceToHost, s->s_query);
    cudaEventRecord(q.ev, s->s_query);
    s->fin_to_wait = q.ev_fin;
    {
        std::lock_guard<std::mutex> ql(s->qmu);
        s->qinflight.push_back(slot);
    }
    s->qcv.notify_one();
    lk.lock();
}

void retire_waves(talp_gpu_server* s) {
    bool any = false;
    while (!s->inflight.empty() && cudaEventQuery(s->inflight.front().ev) == cudaSuccess) {
        Wave& w = s->inflight.front();
        for (int ch : w.chunks) s->free_chunks.push_back(ch);
        if (w.fold) {
            s->slices_folded += w.slices;
            s->records_folded += w.records;
        }
        s->ev_pool.push_back(w.ev);
        s->inflight.pop_front();
        --s->unfinished_waves;
        any = true;
    }
    if (any) {
        s->cv_chunk.notify_all();
        s->cv_done.notify_all();
    }
}

void serve_loop(talp_gpu_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        const uint64_t seen = s->work_gen;
        while (!s->cmds.empty()) {
            Cmd* c = s->cmds.front();
            s->cmds.pop_front();
            if (c->kind == CMD_OPEN)
                c->st = admit(s, c->job, lk, c->msg);
            else
                close_job_locked(s, c, lk);
            c->done = true;
            s->cv_done.notify_all();
        }
        retire_waves(s);
        form_waves(s, lk);
        issue_queries(s, lk);
        if (s->stop && s->inflight.empty() && s->queries.empty() && s->cmds.empty()) break;
        if (!s->inflight.empty()) {
            // waves on the GPU: poll their events at a short period
            s->cv_work.wait_for(lk, std::chrono::microseconds(20), [&] { return s->work_gen != seen; });
        } else {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(5), [&] { return s->work_gen != seen; });
        }
    }
    lk.unlock();
    for (Wave& w : s->inflight) cudaEventSynchronize(w.ev);
    for (Wave& w : s->inflight) cudaEventDestroy(w.ev);
    s->inflight.clear();
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    s->ev_pool.clear();
}

void done_loop(talp_gpu_server* s) {
    cudaSetDevice(s->device);
    while (true) {
        int slot = -1;
        {
            std::unique_lock<std::mutex> ql(s->qmu);
            s->qcv.wait(ql, [&] { return s->stop_done || !s->qinflight.empty(); });
            if (s->qinflight.empty()) return;
            slot = s->qinflight.front();
            s->qinflight.pop_front();
        }
        QSlot& q = s->qslots[slot];
        cudaEventSynchronize(q.ev);
        const Clock::time_point t1 = Clock::now();
        std::lock_guard<std::mutex> lk(s->mu);
        size_t e = 0, et = 0;
        for (Query* r : q.qs) {
            static_assert(sizeof(MetricsOut) == sizeof(talp_gpu_metrics), "metrics record layout");
            static_assert(sizeof(ThreadOut) == sizeof(talp_gpu_thread_tree), "thread tree record layout");
            if (r->tout) {
                memcpy(r->tout, q.h_tout + et, sizeof(ThreadOut) * r->n_out);
                et += r->n_out;
                r->st = check_flags(r->tout, r->n_out);
            } else {
                memcpy(r->out, q.h_out + e, sizeof(MetricsOut) * r->n_out);
                e += r->n_out;
                r->st = check_flags(r->out, r->n_out);
            }
            r->done = true;
            if (s->lat_ms.size() < (1u << 22))
                s->lat_ms.push_back(std::chrono::duration<double, std::milli>(t1 - r->t0).count());
            ++s->queries_answered;
        }
        q.qs.clear();
        q.busy = false;
        s->cv_done.notify_all();
        wake(s);
    }
}

talp_gpu_status fail(talp_gpu_status st, const char* msg) {
    set_last_error(msg);
    return st;
}

}  // namespace

extern "C" {

talp_gpu_status talp_gpu_server_create(talp_gpu_ctx* ctx, const talp_gpu_server_config* cfg, talp_gpu_server** out) {
    if (!ctx || !out) return fail(TALP_GPU_EINVAL, "server_create: null argument");
    *out = nullptr;
    talp_gpu_server* s = new talp_gpu_server();
    s->ctx = ctx;
    s->cfg.max_jobs = cfg && cfg->max_jobs ? cfg->max_jobs : 256;
    s->cfg.max_slice_records = cfg && cfg->max_slice_records ? cfg->max_slice_records : 262144;
    s->cfg.staging_slices = cfg && cfg->staging_slices ? cfg->staging_slices : 64;
    s->device = ctx_device(ctx);
    if (cudaSetDevice(s->device) != cudaSuccess) {
        delete s;
        return fail(TALP_GPU_ECUDA, "server_create: cudaSetDevice failed");
    }
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&s->s_fold, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s->s_query, cudaStreamNonBlocking, hi) != cudaSuccess) {
        talp_gpu_server_destroy(s);
        return fail(TALP_GPU_ECUDA, "server_create: stream creation failed");
    }
    // pinned staging of one slice: 18 bytes per record (raw buffers carry a
    // device index) plus the offsets of the largest job shape
    s->chunk_bytes = align_up(18ull * s->cfg.max_slice_records + 16ull * (kMaxUnitsPerJob + 1) + 256, 4096);
    for (uint32_t k = 0; k < s->cfg.staging_slices; ++k) {
        char* p = nullptr;
        if (cudaMallocHost(&p, s->chunk_bytes) != cudaSuccess) {
            talp_gpu_server_destroy(s);
            return fail(TALP_GPU_ENOMEM, "server_create: pinned staging allocation failed");
        }
        s->chunks.push_back(p);
        s->free_chunks.push_back(static_cast<int>(k));
    }
    s->qslot_entries = static_cast<size_t>(s->cfg.max_jobs) * TALP_GPU_MAX_REGIONS;
    s->qslots.resize(kQuerySlots);
    for (QSlot& q : s->qslots) {
        if (cudaMalloc(&q.d_jobs, sizeof(FinalizeJob) * s->qslot_entries) != cudaSuccess ||
            cudaMalloc(&q.d_out, sizeof(MetricsOut) * s->qslot_entries) != cudaSuccess ||
            cudaMallocHost(&q.h_jobs, sizeof(FinalizeJob) * s->qslot_entries) != cudaSuccess ||
            cudaMallocHost(&q.h_out, sizeof(MetricsOut) * s->qslot_entries) != cudaSuccess ||
            cudaMalloc(&q.d_tjobs, sizeof(ThreadJob) * s->qslot_entries) != cudaSuccess ||
            cudaMalloc(&q.d_tout, sizeof(ThreadOut) * s->qslot_entries) != cudaSuccess ||
            cudaMallocHost(&q.h_tjobs, sizeof(ThreadJob) * s->qslot_entries) != cudaSuccess ||
            cudaMallocHost(&q.h_tout, sizeof(ThreadOut) * s->qslot_entries) != cudaSuccess ||
            cudaEventCreateWithFlags(&q.ev_fin, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&q.ev, cudaEventDisableTiming) != cudaSuccess) {
            talp_gpu_server_destroy(s);
            return fail(TALP_GPU_ENOMEM, "server_create: query buffer allocation failed");
        }
    }
    s->th_serve = std::thread(serve_loop, s);
    s->th_done = std::thread(done_loop, s);
    ctx_hold(ctx, +1);
    s->held = true;
    *out = s;
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_server_open_job(talp_gpu_server* s, uint64_t job_id, uint32_t n_ranks,
                                         const uint32_t* devices_per_rank, uint32_t n_regions,
                                         const int64_t* region_window) {
    if (!s || !devices_per_rank || !region_window || n_ranks == 0 || n_regions == 0 ||
        n_regions > TALP_GPU_MAX_REGIONS)
        return fail(TALP_GPU_EINVAL, "server_open_job: bad argument");
    uint64_t m = 0;
    for (uint32_t i = 0; i < n_ranks; ++i) m += devices_per_rank[i];
    if (n_ranks > kMaxUnitsPerJob || m > kMaxUnitsPerJob)
        return fail(TALP_GPU_EINVAL, "server_open_job: more than 65536 ranks or devices in one job");
    Job* j = new Job();
    j->id = job_id;
    j->n = n_ranks;
    j->m = static_cast<uint32_t>(m);
    j->R = n_regions;
    j->dpr.assign(devices_per_rank, devices_per_rank + n_ranks);
    j->win.assign(region_window, region_window + 2ull * n_regions * n_ranks);
    Cmd c;
    c.kind = CMD_OPEN;
    c.job = j;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop) {
        delete j;
        return fail(TALP_GPU_EBUSY, "server_open_job: server stopping");
    }
    s->cmds.push_back(&c);
    wake(s);
    s->cv_done.wait(lk, [&] { return c.done; });
    if (c.st != TALP_GPU_OK) {
        delete j;
        set_last_error(c.msg);
    }
    return c.st;
}

talp_gpu_status talp_gpu_server_submit(talp_gpu_server* s, uint64_t job_id, const talp_gpu_trace_batch* b) {
    if (!s || !b) return fail(TALP_GPU_EINVAL, "server_submit: null argument");
    if (b->flags & ~static_cast<uint32_t>(TALP_GPU_SORTED_BY_START))
        return fail(TALP_GPU_EINVAL, "server_submit: only TALP_GPU_SORTED_BY_START may be set");
    uint32_t n = 0, m = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return fail(TALP_GPU_ENOTFOUND, "server_submit: unknown job");
        n = it->second->n;
        m = it->second->m;
    }
    if (!b->host_off || !b->dev_off || b->host_off[0] != 0 || b->dev_off[0] != 0)
        return fail(TALP_GPU_EINVAL, "server_submit: offsets must start at 0");
    for (uint32_t i = 0; i < n; ++i)
        if (b->host_off[i + 1] < b->host_off[i]) return fail(TALP_GPU_EINVAL, "server_submit: host_off decreases");
    for (uint32_t g = 0; g < m; ++g)
        if (b->dev_off[g + 1] < b->dev_off[g]) return fail(TALP_GPU_EINVAL, "server_submit: dev_off decreases");
    const uint64_t nh = b->host_off[n], nd = b->dev_off[m];
    if (nh + nd > s->cfg.max_slice_records)
        return fail(TALP_GPU_EINVAL, "server_submit: slice larger than max_slice_records");
    if ((nh && (!b->host_se || !b->host_state)) || (nd && (!b->dev_se || !b->dev_tag)))
        return fail(TALP_GPU_EINVAL, "server_submit: null record array");
    int ch = -1;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_chunk.wait(lk, [&] { return !s->free_chunks.empty() || s->stop; });
        if (s->stop) return fail(TALP_GPU_EBUSY, "server_submit: server stopping");
        ch = s->free_chunks.back();
        s->free_chunks.pop_back();
    }
    // copy the slice into pinned staging (the caller may reuse its memory)
    char* p = s->chunks[ch];
    size_t o = 0;
    auto put = [&](const void* src, size_t bytes) -> char* {
        char* d = p + o;
        if (bytes) memcpy(d, src, bytes);
        o = align_up(o + bytes, 16);
        return d;
    };
    Slice sl;
    sl.chunk = ch;
    sl.flags = b->flags;
    sl.host_se = reinterpret_cast<const int64_t*>(put(b->host_se, 16 * nh));
    sl.dev_se = reinterpret_cast<const int64_t*>(put(b->dev_se, 16 * nd));
    sl.host_state = reinterpret_cast<const uint8_t*>(put(b->host_state, nh));
    sl.dev_tag = reinterpret_cast<const uint8_t*>(put(b->dev_tag, nd));
    sl.host_off = reinterpret_cast<const uint64_t*>(put(b->host_off, 8ull * (n + 1)));
    sl.dev_off = reinterpret_cast<const uint64_t*>(put(b->dev_off, 8ull * (m + 1)));
    sl.records = nh + nd;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) {
        s->free_chunks.push_back(ch);
        s->cv_chunk.notify_all();
        return fail(TALP_GPU_ENOTFOUND, "server_submit: job closed meanwhile");
    }
    it->second->pending.push_back(sl);
    ++it->second->submitted;
    ++s->slices_submitted;
    wake(s);
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_server_submit_raw(talp_gpu_server* s, uint64_t job_id, const talp_gpu_raw_batch* b) {
    if (!s || !b) return fail(TALP_GPU_EINVAL, "server_submit_raw: null argument");
    if (b->flags & ~static_cast<uint32_t>(TALP_GPU_HOLD_BACK))
        return fail(TALP_GPU_EINVAL, "server_submit_raw: only TALP_GPU_HOLD_BACK may be set");
    if ((b->flags & TALP_GPU_HOLD_BACK) && !b->stream_mask)
        return fail(TALP_GPU_EINVAL, "server_submit_raw: hold-back needs the stream masks");
    uint32_t n = 0;
    std::vector<uint32_t> dpr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return fail(TALP_GPU_ENOTFOUND, "server_submit_raw: unknown job");
        n = it->second->n;
        dpr = it->second->dpr;
        for (uint32_t i = 0; i < n; ++i)
            if (dpr[i] > static_cast<uint32_t>(kRawMaxDevices))
                return fail(TALP_GPU_EINVAL, "server_submit_raw: more than 8 devices in a rank");
    }
    if (!b->host_off || !b->raw_off || b->host_off[0] != 0 || b->raw_off[0] != 0)
        return fail(TALP_GPU_EINVAL, "server_submit_raw: offsets must start at 0");
    for (uint32_t i = 0; i < n; ++i)
        if (b->host_off[i + 1] < b->host_off[i] || b->raw_off[i + 1] < b->raw_off[i])
            return fail(TALP_GPU_EINVAL, "server_submit_raw: offsets decrease");
    const uint64_t nh = b->host_off[n], nd = b->raw_off[n];
    if (nh + nd > s->cfg.max_slice_records)
        return fail(TALP_GPU_EINVAL, "server_submit_raw: buffer larger than max_slice_records");
    if ((nh && (!b->host_se || !b->host_state)) || (nd && (!b->raw_se || !b->raw_tag || !b->raw_dev)))
        return fail(TALP_GPU_EINVAL, "server_submit_raw: null record array");
    // A wave folds the raw buffers of many jobs in one call of the raw
    // adapter, which rejects the whole call for one bad record: check the
    // buffer here, so that only its submitter sees the error.  The job's
    // declared streams are the union of every mask it submitted (held
    // records of a stream stay declared).
    std::vector<uint32_t> mask;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return fail(TALP_GPU_ENOTFOUND, "server_submit_raw: unknown job");
        mask = it->second->smask;
        if (dpr.empty()) dpr = it->second->dpr;
    }
    mask.resize(8ull * n, 0u);
    if (b->stream_mask)
        for (uint64_t q = 0; q < 8ull * n; ++q) mask[q] |= b->stream_mask[q];
    const bool hold = (b->flags & TALP_GPU_HOLD_BACK) != 0;
    for (uint32_t i = 0; i < n; ++i)
        for (uint64_t q = b->raw_off[i]; q < b->raw_off[i + 1]; ++q) {
            const uint32_t d = b->raw_dev[q];
            if (d >= dpr[i]) return fail(TALP_GPU_EINVAL, "server_submit_raw: a record names a device its rank does not have");
            if (hold && !((mask[8ull * i + d] >> (b->raw_tag[q] & 31u)) & 1u))
                return fail(TALP_GPU_EINVAL, "server_submit_raw: a record on a stream its device does not declare");
        }
    int ch = -1;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_chunk.wait(lk, [&] { return !s->free_chunks.empty() || s->stop; });
        if (s->stop) return fail(TALP_GPU_EBUSY, "server_submit_raw: server stopping");
        ch = s->free_chunks.back();
        s->free_chunks.pop_back();
    }
    char* p = s->chunks[ch];
    size_t o = 0;
    auto put = [&](const void* src, size_t bytes) -> char* {
        char* d = p + o;
        if (bytes) memcpy(d, src, bytes);
        o = align_up(o + bytes, 16);
        return d;
    };
    Slice sl;
    sl.chunk = ch;
    sl.flags = b->flags;
    sl.raw = true;
    sl.host_se = reinterpret_cast<const int64_t*>(put(b->host_se, 16 * nh));
    sl.dev_se = reinterpret_cast<const int64_t*>(put(b->raw_se, 16 * nd));
    sl.host_state = reinterpret_cast<const uint8_t*>(put(b->host_state, nh));
    sl.dev_tag = reinterpret_cast<const uint8_t*>(put(b->raw_tag, nd));
    sl.raw_dev = reinterpret_cast<const uint8_t*>(put(b->raw_dev, nd));
    sl.host_off = reinterpret_cast<const uint64_t*>(put(b->host_off, 8ull * (n + 1)));
    sl.dev_off = reinterpret_cast<const uint64_t*>(put(b->raw_off, 8ull * (n + 1)));
    sl.records = nh + nd;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) {
        s->free_chunks.push_back(ch);
        s->cv_chunk.notify_all();
        return fail(TALP_GPU_ENOTFOUND, "server_submit_raw: job closed meanwhile");
    }
    std::vector<uint32_t>& sm = it->second->smask;
    sm.resize(8ull * n, 0u);
    if (b->stream_mask)
        for (uint64_t q = 0; q < 8ull * n; ++q) sm[q] |= b->stream_mask[q];
    it->second->pending.push_back(sl);
    ++it->second->submitted;
    ++s->slices_submitted;
    wake(s);
    return TALP_GPU_OK;
}

static talp_gpu_status server_query_common(talp_gpu_server* s, uint64_t job_id, uint32_t region,
                                           talp_gpu_metrics* out, talp_gpu_thread_tree* tout,
                                           const uint32_t* proc_off, uint32_t n_procs) {
    Query q;
    q.job = job_id;
    q.region = region;
    q.out = out;
    q.tout = tout;
    q.proc_off = proc_off;
    q.n_procs = n_procs;
    q.t0 = Clock::now();
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(TALP_GPU_ENOTFOUND, "server_query: unknown job");
    if (region != TALP_GPU_ALL_REGIONS && region >= it->second->R)
        return fail(TALP_GPU_EINVAL, "server_query: region out of range");
    if (tout) {
        if (n_procs == 0 || proc_off[0] != 0 || proc_off[n_procs] != it->second->n)
            return fail(TALP_GPU_EINVAL, "server_query_threads: proc_off must run from 0 to the job's n_ranks");
        for (uint32_t i = 0; i < n_procs; ++i)
            if (proc_off[i + 1] <= proc_off[i])
                return fail(TALP_GPU_EINVAL, "server_query_threads: a process without threads in proc_off");
    }
    q.n_out = region == TALP_GPU_ALL_REGIONS ? it->second->R : 1;
    q.need = it->second->submitted;
    s->queries.push_back(&q);
    wake(s);
    s->cv_done.wait(lk, [&] { return q.done; });
    if (q.st == TALP_GPU_ENOTFOUND)
        set_last_error("server_query: job closed");
    else if (q.st == TALP_GPU_ETIMEDOUT)
        set_last_error("server_query: a device wait timed out");
    else if (q.st == TALP_GPU_ENOMEM)
        set_last_error("server_query_threads: no memory for the process table");
    else if (q.st != TALP_GPU_OK)
        set_last_error("server_query: the job holds invalid or out-of-order records");
    return q.st;
}

talp_gpu_status talp_gpu_server_query(talp_gpu_server* s, uint64_t job_id, uint32_t region,
                                      talp_gpu_metrics* out_host) {
    if (!s || !out_host) return fail(TALP_GPU_EINVAL, "server_query: null argument");
    return server_query_common(s, job_id, region, out_host, nullptr, nullptr, 0);
}

talp_gpu_status talp_gpu_server_query_threads(talp_gpu_server* s, uint64_t job_id, uint32_t region,
                                              const uint32_t* proc_off, uint32_t n_procs,
                                              talp_gpu_thread_tree* out_host) {
    if (!s || !out_host || !proc_off) return fail(TALP_GPU_EINVAL, "server_query_threads: null argument");
    return server_query_common(s, job_id, region, nullptr, out_host, proc_off, n_procs);
}

talp_gpu_status talp_gpu_server_drain(talp_gpu_server* s) {
    if (!s) return fail(TALP_GPU_EINVAL, "server_drain: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] {
        for (auto& kv : s->jobs)
            if (!kv.second->pending.empty() && kv.second->error == TALP_GPU_OK) return false;
        return s->unfinished_waves == 0;
    });
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_server_close_job(talp_gpu_server* s, uint64_t job_id) {
    if (!s) return fail(TALP_GPU_EINVAL, "server_close_job: null server");
    Cmd c;
    c.kind = CMD_CLOSE;
    c.id = job_id;
    std::unique_lock<std::mutex> lk(s->mu);
    // fold what the job still has queued, then close it
    s->cv_done.wait(lk, [&] {
        auto it = s->jobs.find(job_id);
        return it == s->jobs.end() || it->second->pending.empty() || it->second->error != TALP_GPU_OK;
    });
    s->cmds.push_back(&c);
    wake(s);
    s->cv_done.wait(lk, [&] { return c.done; });
    if (c.st != TALP_GPU_OK) set_last_error(c.msg);
    return c.st;
}

talp_gpu_status talp_gpu_server_info(talp_gpu_server* s, talp_gpu_server_stats* out) {
    if (!s || !out) return fail(TALP_GPU_EINVAL, "server_info: null argument");
    std::vector<double> v;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        memset(out, 0, sizeof(*out));
        out->slices_submitted = s->slices_submitted;
        out->slices_folded = s->slices_folded;
        out->records_folded = s->records_folded;
        out->waves = s->waves;
        out->queries = s->queries_answered;
        out->query_batches = s->query_batches;
        out->jobs_open = static_cast<uint32_t>(s->jobs.size());
        v = s->lat_ms;
    }
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        // nearest-rank percentiles
        auto pct = [&](double p) {
            const size_t r = static_cast<size_t>(p * static_cast<double>(v.size()) + 0.999999);
            return v[std::min(v.size(), std::max<size_t>(r, 1)) - 1];
        };
        out->query_p50_ms = pct(0.50);
        out->query_p99_ms = pct(0.99);
        out->query_max_ms = v.back();
    }
    return TALP_GPU_OK;
}

talp_gpu_status talp_gpu_server_destroy(talp_gpu_server* s) {
    if (!s) return TALP_GPU_OK;
    if (s->th_serve.joinable()) {
        std::vector<uint64_t> ids;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (auto& kv : s->jobs) ids.push_back(kv.first);
        }
        for (uint64_t id : ids) talp_gpu_server_close_job(s, id);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
            wake(s);
        }
        s->cv_chunk.notify_all();
        s->th_serve.join();
    }
    if (s->th_done.joinable()) {
        {
            std::lock_guard<std::mutex> ql(s->qmu);
            s->stop_done = true;
        }
        s->qcv.notify_all();
        s->th_done.join();
    }
    cudaSetDevice(s->device);
    for (char* p : s->chunks) cudaFreeHost(p);
    for (QSlot& q : s->qslots) {
        if (q.d_jobs) cudaFree(q.d_jobs);
        if (q.d_out) cudaFree(q.d_out);
        if (q.h_jobs) cudaFreeHost(q.h_jobs);
        if (q.h_out) cudaFreeHost(q.h_out);
        if (q.d_tjobs) cudaFree(q.d_tjobs);
        if (q.d_tout) cudaFree(q.d_tout);
        if (q.h_tjobs) cudaFreeHost(q.h_tjobs);
        if (q.h_tout) cudaFreeHost(q.h_tout);
        if (q.d_po) cudaFree(q.d_po);
        if (q.h_po) cudaFreeHost(q.h_po);
        if (q.ev_fin) cudaEventDestroy(q.ev_fin);
        if (q.ev) cudaEventDestroy(q.ev);
    }
    if (s->s_fold) cudaStreamDestroy(s->s_fold);
    if (s->s_query) cudaStreamDestroy(s->s_query);
    if (s->held) ctx_hold(s->ctx, -1);
    delete s;
    return TALP_GPU_OK;
}

}  // extern "C"
