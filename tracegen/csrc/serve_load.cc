// Client load of the serving workload, in native threads: submitter threads
// with Poisson arrivals queue time slices of their jobs, query threads ask
// every job of theirs for all its regions once per query period, and each
// query's latency is taken around the call.  The calls go straight to the
// library's C ABI (its entry points are passed in as function pointers, so
// that this file links to no particular build of the library), the way an
// instrumented application asks for metrics at run time (Sec. 3.2).
//
// A job's slices are a fixed list cycled with a time shift: slice q is list
// entry q % n_slices with every host and device timestamp moved by
// (q / n_slices) * span, which keeps each device's records in time order
// from one cycle to the next.
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <random>
#include <thread>
#include <vector>

#include "talp_gpu.h"

namespace {

using Clock = std::chrono::steady_clock;
using SubmitFn = talp_gpu_status (*)(talp_gpu_server*, uint64_t, const talp_gpu_trace_batch*);
using QueryFn = talp_gpu_status (*)(talp_gpu_server*, uint64_t, uint32_t, talp_gpu_metrics*);

}  // namespace

extern "C" {

typedef struct {
    uint64_t job_id;
    uint32_t n_ranks, n_devices;          // rows of host_off and dev_off: n + 1 entries
    uint32_t n_slices, n_regions;
    int64_t span;                         // time shift per cycle through the slices
    const talp_gpu_trace_batch* slices;   // [n_slices], host record arrays
} sl_job;

typedef struct {
    double rate;        // slice arrivals per second over all submitters (Poisson)
    double query_s;     // query period of every job
    double seconds;     // length of the run
    uint32_t n_sub, n_q;
    uint64_t seed;
} sl_config;

typedef struct {
    uint64_t slices, records;   // submitted
    uint64_t queries;           // answered (latencies written: min(queries, lat_cap))
    uint64_t errors;
    int32_t first_error;        // talp_gpu_status of the first failed call, 0 if none
    int32_t reserved;
    double wall_s;
} sl_result;

// Runs the load for cfg->seconds.  next_q[n_jobs] is each job's next slice
// number (read and advanced).  Returns 0, or -1 for bad arguments.
int sl_run(void* srv_p, void* submit_p, void* query_p, const sl_job* jobs, uint32_t n_jobs, uint64_t* next_q,
           const sl_config* cfg, double* lat_out, uint64_t lat_cap, sl_result* res) {
    if (!srv_p || !submit_p || !query_p || !jobs || !next_q || !cfg || !res || n_jobs == 0 || cfg->n_sub == 0 ||
        cfg->n_q == 0 || cfg->rate <= 0.0 || cfg->query_s <= 0.0)
        return -1;
    auto* srv = static_cast<talp_gpu_server*>(srv_p);
    const SubmitFn submit = reinterpret_cast<SubmitFn>(submit_p);
    const QueryFn query = reinterpret_cast<QueryFn>(query_p);
    std::atomic<bool> stop{false};
    std::atomic<uint64_t> slices{0}, records{0}, errors{0};
    std::atomic<int32_t> first_error{0};
    std::mutex lat_mu;
    std::vector<double> lat_all;
    uint32_t max_regions = 1;
    for (uint32_t j = 0; j < n_jobs; ++j) max_regions = jobs[j].n_regions > max_regions ? jobs[j].n_regions : max_regions;
    auto fail = [&](talp_gpu_status st) {
        errors.fetch_add(1);
        int32_t z = 0;
        first_error.compare_exchange_strong(z, static_cast<int32_t>(st));
    };

    auto submitter = [&](uint32_t tid) {
        std::mt19937_64 rng(cfg->seed * 1000003ull + tid);
        std::exponential_distribution<double> gap(cfg->rate / cfg->n_sub);
        std::vector<uint32_t> mine;
        for (uint32_t j = tid; j < n_jobs; j += cfg->n_sub) mine.push_back(j);
        if (mine.empty()) return;
        std::uniform_int_distribution<size_t> pick(0, mine.size() - 1);
        std::vector<int64_t> hbuf, dbuf;
        auto t_next = Clock::now();
        while (!stop.load(std::memory_order_relaxed)) {
            t_next += std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(gap(rng)));
            std::this_thread::sleep_until(t_next);
            if (stop.load(std::memory_order_relaxed)) break;
            const uint32_t j = mine[pick(rng)];
            const sl_job& J = jobs[j];
            const uint64_t q = next_q[j];
            const talp_gpu_trace_batch& base = J.slices[q % J.n_slices];
            const int64_t shift = static_cast<int64_t>(q / J.n_slices) * J.span;
            const uint64_t nh = base.host_off[J.n_ranks], nd = base.dev_off[J.n_devices];
            talp_gpu_trace_batch b = base;
            if (shift != 0) {
                hbuf.resize(2 * nh);
                dbuf.resize(2 * nd);
                for (uint64_t i = 0; i < 2 * nh; ++i) hbuf[i] = base.host_se[i] + shift;
                for (uint64_t i = 0; i < 2 * nd; ++i) dbuf[i] = base.dev_se[i] + shift;
                b.host_se = hbuf.data();
                b.dev_se = dbuf.data();
            }
            const talp_gpu_status st = submit(srv, J.job_id, &b);
            if (st != TALP_GPU_OK) {
                fail(st);
                break;
            }
            next_q[j] = q + 1;
            slices.fetch_add(1, std::memory_order_relaxed);
            records.fetch_add(nh + nd, std::memory_order_relaxed);
        }
    };

    auto querier = [&](uint32_t tid) {
        std::vector<uint32_t> mine;
        for (uint32_t j = tid; j < n_jobs; j += cfg->n_q) mine.push_back(j);
        std::vector<talp_gpu_metrics> out(max_regions);
        std::vector<double> lat;
        const auto period = std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(cfg->query_s));
        auto t_tick = Clock::now();
        bool ok = true;
        while (ok && !stop.load(std::memory_order_relaxed)) {
            for (uint32_t j : mine) {
                const auto q0 = Clock::now();
                const talp_gpu_status st = query(srv, jobs[j].job_id, TALP_GPU_ALL_REGIONS, out.data());
                lat.push_back(std::chrono::duration<double>(Clock::now() - q0).count());
                if (st != TALP_GPU_OK) {
                    fail(st);
                    ok = false;
                    break;
                }
            }
            t_tick += period;
            if (t_tick > Clock::now())
                std::this_thread::sleep_until(t_tick);
            else
                t_tick = Clock::now();
        }
        std::lock_guard<std::mutex> g(lat_mu);
        lat_all.insert(lat_all.end(), lat.begin(), lat.end());
    };

    const auto w0 = Clock::now();
    std::vector<std::thread> th;
    for (uint32_t i = 0; i < cfg->n_sub; ++i) th.emplace_back(submitter, i);
    for (uint32_t i = 0; i < cfg->n_q; ++i) th.emplace_back(querier, i);
    std::this_thread::sleep_for(std::chrono::duration<double>(cfg->seconds));
    stop.store(true);
    for (auto& x : th) x.join();
    res->wall_s = std::chrono::duration<double>(Clock::now() - w0).count();
    res->slices = slices.load();
    res->records = records.load();
    res->queries = lat_all.size();
    res->errors = errors.load();
    res->first_error = first_error.load();
    res->reserved = 0;
    const uint64_t n = lat_all.size() < lat_cap ? lat_all.size() : lat_cap;
    if (lat_out && n) std::memcpy(lat_out, lat_all.data(), n * sizeof(double));
    return 0;
}

}  // extern "C"
