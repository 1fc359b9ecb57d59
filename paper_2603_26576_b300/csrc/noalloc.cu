// talp_gpu_reduce_noalloc: the whole reduction of one trace without any
// device allocation, for callers that must not call cudaMalloc/cudaFree.
//
// Typical such callers are monitoring hooks that live inside the
// application being measured: the application (or its framework's caching
// allocator) owns the device memory and may have reserved all of it, and a
// cudaMalloc or cudaFree issued from the hook could fail or synchronise the
// device and stall the application's own streams.  This entry point needs no
// context and allocates nothing: its scratch (segment table, per-unit
// partial sums, windows, running carries, warp records, metrics) lives in a
// file-scope __device__ array of fixed size.
//
// Limits: n_ranks + m <= TALP_GPU_NOALLOC_MAX_UNITS units, n_regions <= 8,
// device record arrays already in start order (no sort scratch).
//
// Sharing: every call on a device uses that device's one copy of the array,
// which keeps the last call's contents; every call clears what must start at
// zero.  Two calls whose GPU work overlapped would race on it, so a call
// holds a per-device lock from its first enqueue until its stream has
// finished the work (on error paths too): calls made through this library in
// one process never overlap on a device.
//
// Module loading: under CUDA's default lazy loading the array and the
// kernels' code are loaded on the first call on each device, which is a
// device allocation made by the driver.  Every call launches the same
// kernels (also for a trace without records), so one first call during
// set-up -- before the application fills the device's memory and before
// any stream capture -- leaves nothing to load later.
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/talp_gpu.h"
#include "kernels.h"

using namespace talp;

namespace {

constexpr uint32_t kMaxUnits = TALP_GPU_NOALLOC_MAX_UNITS;
constexpr uint32_t kMaxR = TALP_GPU_MAX_REGIONS;
constexpr uint32_t kMaxWarps = 4096;
constexpr uint32_t kMaxJobs = 16;
constexpr uint32_t kMaxDevices = 64;

constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }

// scratch layout (byte offsets); the first part is uploaded from the host
constexpr size_t kOffSegs = 0;
constexpr size_t kOffStart = al(kOffSegs + sizeof(SegDesc) * kMaxUnits);
constexpr size_t kOffEnd = al(kOffStart + sizeof(uint64_t) * (kMaxUnits + 1));
constexpr size_t kOffJobs = al(kOffEnd + sizeof(uint64_t) * (kMaxUnits + 1));
constexpr size_t kOffFin = al(kOffJobs + sizeof(FillJob) * kMaxJobs);
constexpr size_t kOffWin = al(kOffFin + sizeof(FinalizeJob) * kMaxR);
constexpr size_t kOffRank = al(kOffWin + sizeof(int64_t) * 2 * kMaxR * kMaxUnits);
constexpr size_t kOffTdev = al(kOffRank + sizeof(int64_t) * kMaxUnits);
constexpr size_t kUploadBytes = al(kOffTdev + sizeof(TraceDev));
// device-only part
constexpr size_t kOffHsum = kUploadBytes;
constexpr size_t kOffDsum = al(kOffHsum + sizeof(int64_t) * 3 * kMaxR * kMaxUnits);
constexpr size_t kOffCarry = al(kOffDsum + sizeof(int64_t) * 3 * kMaxR * kMaxUnits);
constexpr size_t kOffCarry2 = al(kOffCarry + sizeof(int64_t) * 3 * kMaxUnits);
constexpr size_t kOffStatus = al(kOffCarry2 + sizeof(int64_t) * 3 * kMaxUnits);
constexpr size_t kOffGstatus = kOffStatus + 256;
constexpr size_t kOffFlags = kOffGstatus + 256;
constexpr size_t kOffWrec = al(kOffFlags + sizeof(uint32_t) * (kMaxUnits + 2));
constexpr size_t kOffMetrics = al(kOffWrec + sizeof(WarpRec) * kMaxWarps);
constexpr size_t kScratchBytes = al(kOffMetrics + sizeof(MetricsOut) * kMaxR);

static_assert(kScratchBytes <= (6u << 20), "no-alloc scratch stays within 6 MiB");

// The scratch.  Host code must not use this name as a device address: each
// device's address comes from cudaGetSymbolAddress at set-up.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host copy of the uploaded part (pageable; cudaMemcpyAsync from pageable
// memory has consumed the source when it returns).  One copy serves every
// device: g_stage_mu is held while it is filled and copied.
static unsigned char g_host_stage[kUploadBytes];
std::mutex g_stage_mu;

// Per device: the lock held through a call's GPU work, and the scratch's
// device address with the id of the context it was looked up in (a device
// reset makes a new primary context, in which the array has a new address).
struct DevSlot {
    std::mutex mu;
    unsigned char* scratch = nullptr;
    unsigned long long ctx_id = 0;
};
DevSlot g_dev[kMaxDevices];

// Driver calls reached through the runtime's entry-point query (the library
// does not link the driver library itself).
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

// Id of the calling thread's current context; 0 when it cannot be had.
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
    });
    if (!get_cur || !get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device-side wait limit in clock cycles: TALP_GPU_WAIT_LIMIT as for
// contexts (a negative value reports a time-out at once), else ~2 s.
int64_t wait_limit_cycles() {
    if (const char* s = getenv("TALP_GPU_WAIT_LIMIT")) return strtoll(s, nullptr, 10);
    return 4000000000LL;
}

talp_gpu_status err(talp_gpu_status st, const char* msg) {
    set_last_error(msg);
    return st;
}

}  // namespace

extern "C" talp_gpu_status talp_gpu_reduce_noalloc(const talp_gpu_trace_batch* b, talp_gpu_metrics* out_host,
                                                  void* stream_) {
    if (!b || !out_host) return err(TALP_GPU_EINVAL, "null argument");
    const uint32_t need = TALP_GPU_DEVICE_PTRS | TALP_GPU_SORTED_BY_START;
    if (b->flags != need || b->reserved)
        return err(TALP_GPU_EINVAL,
                   "no-alloc reduction takes exactly DEVICE_PTRS | SORTED_BY_START (device records in start order)");
    if (b->n_ranks == 0 || b->n_regions == 0 || b->n_regions > kMaxR)
        return err(TALP_GPU_EINVAL, "n_ranks >= 1 and 1 <= n_regions <= 8");
    if (!b->devices_per_rank || !b->region_window || !b->host_off || !b->dev_off)
        return err(TALP_GPU_EINVAL, "null header array");
    uint64_t m64 = 0;
    for (uint32_t i = 0; i < b->n_ranks; ++i) m64 += b->devices_per_rank[i];
    if (b->n_ranks + m64 > kMaxUnits)
        return err(TALP_GPU_EINVAL, "no-alloc reduction: n_ranks + devices exceeds TALP_GPU_NOALLOC_MAX_UNITS");
    const uint32_t n = b->n_ranks, m = static_cast<uint32_t>(m64), R = b->n_regions;
    if (b->host_off[0] != 0 || b->dev_off[0] != 0) return err(TALP_GPU_EINVAL, "offsets must start at 0");
    for (uint32_t i = 0; i < n; ++i)
        if (b->host_off[i + 1] < b->host_off[i]) return err(TALP_GPU_EINVAL, "host_off not monotone");
    for (uint32_t g = 0; g < m; ++g)
        if (b->dev_off[g + 1] < b->dev_off[g]) return err(TALP_GPU_EINVAL, "dev_off not monotone");
    for (uint64_t k = 0; k < 2ull * R * n; k += 2)
        if (b->region_window[k + 1] < b->region_window[k]) return err(TALP_GPU_EINVAL, "window end < begin");
    const uint64_t nh = b->host_off[n], nd = b->dev_off[m];
    if ((nh && (!b->host_se || !b->host_state)) || (nd && (!b->dev_se || !b->dev_tag)))
        return err(TALP_GPU_EINVAL, "null record array");
    auto mis = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
    if ((nh && (mis(b->host_se) || mis(b->host_state))) || (nd && (mis(b->dev_se) || mis(b->dev_tag))))
        return err(TALP_GPU_EINVAL, "device record arrays must be 16-byte aligned");

    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= static_cast<int>(kMaxDevices))
        return err(TALP_GPU_ECUDA, "cudaGetDevice");

    DevSlot& slot = g_dev[dev];
    std::lock_guard<std::mutex> lock(slot.mu);
    // set-up, once per device (again after a device reset made a new
    // context), with that device current: the scratch's device address.  The
    // first call on a device does this; make it before any stream capture.
    const unsigned long long ctx_id = current_ctx_id();
    if (!slot.scratch || ctx_id != slot.ctx_id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return err(TALP_GPU_ECUDA, "cudaGetSymbolAddress of the no-alloc scratch");
        slot.scratch = static_cast<unsigned char*>(p);
        slot.ctx_id = ctx_id;
    }
    unsigned char* S = slot.scratch;
    std::unique_lock<std::mutex> stage_lock(g_stage_mu);
    unsigned char* H = g_host_stage;

    SegDesc* sd = reinterpret_cast<SegDesc*>(H + kOffSegs);
    uint64_t* sstart = reinterpret_cast<uint64_t*>(H + kOffStart);
    uint64_t* send = reinterpret_cast<uint64_t*>(H + kOffEnd);
    FillJob* jobs = reinterpret_cast<FillJob*>(H + kOffJobs);
    FinalizeJob* fin = reinterpret_cast<FinalizeJob*>(H + kOffFin);
    int64_t* hwin_h = reinterpret_cast<int64_t*>(H + kOffWin);
    int64_t* rank_h = reinterpret_cast<int64_t*>(H + kOffRank);
    int64_t* hsum = reinterpret_cast<int64_t*>(S + kOffHsum);
    int64_t* dsum = reinterpret_cast<int64_t*>(S + kOffDsum);
    int64_t* hwin = reinterpret_cast<int64_t*>(S + kOffWin);
    int64_t* cin = reinterpret_cast<int64_t*>(S + kOffCarry);
    int64_t* cout = reinterpret_cast<int64_t*>(S + kOffCarry2);
    uint32_t* status = reinterpret_cast<uint32_t*>(S + kOffStatus);
    uint32_t* gstatus = reinterpret_cast<uint32_t*>(S + kOffGstatus);
    uint32_t* flags = reinterpret_cast<uint32_t*>(S + kOffFlags);
    WarpRec* wrec = reinterpret_cast<WarpRec*>(S + kOffWrec);
    MetricsOut* mout = reinterpret_cast<MetricsOut*>(S + kOffMetrics);
    TraceDev* tdev = reinterpret_cast<TraceDev*>(S + kOffTdev);

    for (uint32_t i = 0; i < n; ++i)
        for (uint32_t r = 0; r < R; ++r) {
            hwin_h[(i * R + r) * 2 + 0] = b->region_window[(static_cast<size_t>(r) * n + i) * 2 + 0];
            hwin_h[(i * R + r) * 2 + 1] = b->region_window[(static_cast<size_t>(r) * n + i) * 2 + 1];
        }
    {
        uint32_t g = 0;
        for (uint32_t i = 0; i < n; ++i)
            for (uint32_t q = 0; q < b->devices_per_rank[i]; ++q) rank_h[g++] = i;
    }
    TraceDev td{};
    td.trace_id = b->trace_id;
    td.n = n;
    td.m = m;
    td.R = R;
    td.hsum = hsum;
    td.dsum = dsum;
    td.hwin = hwin;
    td.dev_rank = reinterpret_cast<const int64_t*>(S + kOffRank);
    td.status = status;
    memcpy(H + kOffTdev, &td, sizeof(TraceDev));

    const uint8_t* hlim = reinterpret_cast<const uint8_t*>(
        reinterpret_cast<uintptr_t>(b->host_state + nh) & ~static_cast<uintptr_t>(15));
    const uint8_t* dlim = reinterpret_cast<const uint8_t*>(
        reinterpret_cast<uintptr_t>(b->dev_tag + nd) & ~static_cast<uintptr_t>(15));
    // virtual positions: records plus a fixed cost per segment (balances
    // segment switches across warps)
    const uint64_t seg_cost = 512 + 64ull * R + 2ull * (R - 1) * static_cast<uint64_t>(sweep_tile(kDefaultSweepShape));
    uint64_t pos = 0, nrec = 0;
    uint32_t si = 0;
    for (uint32_t g = 0; g < m; ++g, ++si) {
        SegDesc& s = sd[si];
        memset(&s, 0, sizeof(SegDesc));
        const uint64_t o = b->dev_off[g];
        s.se = b->dev_se + 2 * o;
        s.tag = b->dev_tag + o;
        s.tag_limit = dlim;
        s.sums = dsum + static_cast<size_t>(g) * R * 3;
        s.win = hwin + static_cast<size_t>(rank_h[g]) * R * 2;
        s.status = status;
        s.carry_in = cin + 3ull * g;
        s.carry_out = cout + 3ull * g;
        s.n = b->dev_off[g + 1] - o;
        s.R = static_cast<uint16_t>(R);
        s.is_host = 0;
        sstart[si] = pos;
        send[si] = pos + s.n;
        pos += s.n + seg_cost;
        nrec += s.n;
    }
    for (uint32_t i = 0; i < n; ++i, ++si) {
        SegDesc& s = sd[si];
        memset(&s, 0, sizeof(SegDesc));
        const uint64_t o = b->host_off[i];
        s.se = b->host_se + 2 * o;
        s.tag = b->host_state + o;
        s.tag_limit = hlim;
        s.sums = hsum + static_cast<size_t>(i) * R * 3;
        s.win = hwin + static_cast<size_t>(i) * R * 2;
        s.status = status;
        s.n = b->host_off[i + 1] - o;
        s.R = static_cast<uint16_t>(R);
        s.is_host = 1;
        sstart[si] = pos;
        send[si] = pos + s.n;
        pos += s.n + seg_cost;
        nrec += s.n;
    }
    sstart[si] = pos;
    send[si] = pos;
    const uint32_t n_segs = si;

    // what must start at zero (the array keeps the previous call's contents)
    uint32_t nj = 0;
    jobs[nj++] = FillJob{hsum, 3ull * n * R, 0, nullptr};
    if (m) jobs[nj++] = FillJob{dsum, 3ull * m * R, 0, nullptr};
    if (m) jobs[nj++] = FillJob{cin, 3ull * m, NEG_INF, nullptr};
    if (m) jobs[nj++] = FillJob{cout, 3ull * m, NEG_INF, nullptr};
    jobs[nj++] = FillJob{reinterpret_cast<int64_t*>(status), 1, 0, nullptr};
    jobs[nj++] = FillJob{reinterpret_cast<int64_t*>(gstatus), 1, 0, nullptr};
    jobs[nj++] = FillJob{reinterpret_cast<int64_t*>(flags), (n_segs + 2) / 2, 0, nullptr};
    for (uint32_t r = 0; r < R; ++r) fin[r] = FinalizeJob{tdev, mout + r, r, 0};

    // sweep grid, capped by the warp records the scratch holds
    const int shape = kDefaultSweepShape;
    const int tile = sweep_tile(shape);
    const int warps = kSweepShapes[shape].warps;
    const int cps = sweep_ctas_per_sm(shape, static_cast<int>(R));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cps <= 0 || sms <= 0) return err(TALP_GPU_ECUDA, "sweep kernel cannot be resident");
    uint64_t want = ((pos + tile - 1) / tile + 3) / 4;
    uint64_t maxw = static_cast<uint64_t>(sms) * cps * warps;
    if (maxw > kMaxWarps) maxw = kMaxWarps / warps * warps;
    if (want > maxw) want = maxw;
    if (want < 1) want = 1;
    const int grid = static_cast<int>((want + warps - 1) / warps);
    const uint32_t n_wrec = static_cast<uint32_t>(grid) * warps;

    // Every kernel is launched whatever the record count (the sweep and the
    // fix-up return at once without records), so that any first call loads
    // all of this entry point's device code.
    const int64_t wait_limit = wait_limit_cycles();
    cudaError_t e = cudaMemcpyAsync(S, H, kUploadBytes, cudaMemcpyHostToDevice, stream);
    stage_lock.unlock();   // a copy from pageable memory has consumed its source when it returns
    bool enqueued = e == cudaSuccess;
    if (e == cudaSuccess) e = launch_prep(reinterpret_cast<const FillJob*>(S + kOffJobs), nj, stream);
    if (e == cudaSuccess)
        e = launch_sweep(shape, static_cast<int>(R), grid, reinterpret_cast<const SegDesc*>(S + kOffSegs),
                         reinterpret_cast<const uint64_t*>(S + kOffStart),
                         reinterpret_cast<const uint64_t*>(S + kOffEnd), n_segs, wrec, flags, gstatus, wait_limit,
                         false, RunLog{nullptr, nullptr}, 0u, nullptr, stream);
    if (e == cudaSuccess)
        e = launch_fixup(reinterpret_cast<const SegDesc*>(S + kOffSegs),
                         reinterpret_cast<const uint64_t*>(S + kOffStart), wrec, n_wrec, flags, false,
                         RunLog{nullptr, nullptr}, stream);
    if (e == cudaSuccess) e = launch_finalize(reinterpret_cast<const FinalizeJob*>(S + kOffFin), R, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_host, mout, sizeof(MetricsOut) * R, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        // work already queued still reads the scratch: let it finish before
        // the lock goes, so that the next call cannot overwrite it underneath
        if (enqueued) (void)cudaStreamSynchronize(stream);
        set_last_error(std::string("no-alloc reduction: ") + cudaGetErrorString(e));
        return TALP_GPU_ECUDA;
    }
    for (uint32_t r = 0; r < R; ++r) {
        if (out_host[r].flags & TALP_GPU_M_TIMEOUT) return err(TALP_GPU_ETIMEDOUT, "a device-side wait ran out");
        if (out_host[r].flags & (TALP_GPU_M_INVALID | TALP_GPU_M_UNSORTED))
            return err(TALP_GPU_EINVAL, "invalid or out-of-order records");
    }
    return TALP_GPU_OK;
}
