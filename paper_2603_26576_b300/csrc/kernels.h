// Launchers of the reducer's kernels (host-callable; used by the engine).
#pragma once
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "common.cuh"

namespace talp {

// Shape of the sweep kernel: records per lane per tile (odd, so that the
// blocked shared-memory reads are free of bank conflicts), warps per CTA and
// TMA pipeline stages per warp.
struct SweepShape {
    int items;
    int warps;
    int stages;
};

constexpr int kNumSweepShapes = 4;
constexpr int kDefaultSweepShape = 3;   // fastest on the large single-trace workload
extern const SweepShape kSweepShapes[kNumSweepShapes];

// Largest number of co-resident CTAs per SM for a shape, 0 if it cannot run.
int sweep_ctas_per_sm(int shape, int rmax);
int sweep_tile(int shape);

// seg_start[s]: virtual start of segment s (n_segs + 1 entries, the last the
// total); seg_rend[s]: virtual end of its records (start + records).  The
// gap up to seg_start[s + 1] is the segment's share of fixed cost.
// ticket null: one slice of the virtual array per warp (wrec: grid * warps
// records); else n_slices slices handed out through *ticket, which must be
// 0 at launch (wrec: n_slices records).
cudaError_t launch_sweep(int shape, int rmax, int grid, const SegDesc* segs, const uint64_t* seg_start,
                         const uint64_t* seg_rend, uint32_t n_segs, WarpRec* wrec, uint32_t* seg_flags,
                         uint32_t* gstatus, int64_t wait_limit, bool skip_sorted_out, RunLog rl,
                         uint32_t n_slices, uint32_t* ticket, cudaStream_t stream);

// rl: the run log the first sweep (skip_sorted_out) fills, or {null, null}
cudaError_t launch_fixup(const SegDesc* segs, const uint64_t* seg_start, const WarpRec* wrec, uint32_t n_wrec,
                         uint32_t* seg_flags, bool skip_resorted, RunLog rl, cudaStream_t stream);

cudaError_t launch_prep(const FillJob* jobs, uint32_t n_jobs, cudaStream_t stream);

cudaError_t launch_finalize(const FinalizeJob* jobs, uint32_t n_jobs, cudaStream_t stream);
cudaError_t launch_thread_tree(const ThreadJob* jobs, uint32_t n_jobs, cudaStream_t stream);
cudaError_t launch_thread_combine(const ThreadOut* parts, uint32_t n_parts, ThreadOut* out, cudaStream_t stream);
cudaError_t launch_concurrency(const int64_t* se, const uint8_t* tag, const ConcDev* devs, uint32_t n_dev,
                               const ConcChunk* chunks, uint32_t n_chunks, int64_t* top, int64_t* in, int64_t* snap,
                               int64_t* out, uint32_t* status, cudaStream_t stream);
cudaError_t launch_raw_count(const RawTile* tiles, uint32_t n_tiles, const RawRank* ranks, uint32_t n_ranks,
                             uint32_t* hist, uint64_t* offs, RawMove* moves, uint64_t* dev_count,
                             uint32_t* dev_streams, uint64_t* dev_runs, uint32_t* status, int grid,
                             cudaStream_t stream);
cudaError_t launch_raw_scatter(const RawTile* tiles, uint32_t n_tiles, const RawRank* ranks, const uint64_t* offs,
                               int64_t* lse, uint8_t* ltag, uint32_t* status, int64_t wait_limit, int grid,
                               cudaStream_t stream);
cudaError_t launch_raw_hold(const RawRank* ranks, uint32_t n_ranks, const int64_t* lse, RawMove* moves,
                            uint64_t* fold_count, uint64_t* hold_count, uint32_t* status, uint64_t* dev_runs,
                            cudaStream_t stream);
cudaError_t launch_raw_move(const RawTile* tiles, uint32_t n_tiles, const RawRank* ranks, const RawMove* moves,
                            const uint64_t* fold_base, const int64_t* lse, const uint8_t* ltag, int64_t* fse,
                            uint8_t* ftag, int grid, cudaStream_t stream);
int raw_tile_records();
cudaError_t launch_scalability(const MetricsOut* runs, uint32_t n_runs, uint32_t ref, int weak, ScaleOut* out,
                               cudaStream_t stream);
cudaError_t launch_combine(const MetricsOut* parts, uint32_t n_parts, MetricsOut* out, cudaStream_t stream);

// Sort stage over the device segments flagged out of order (sortable ones):
// segments of a few sorted runs are merged and swept at once (fused
// merge-sweep), the others radix sorted; then the segment table of the
// sorted copies for the re-sweep.
// n_segs: entries of `segs`; n_slots: device segments (upper bound of flagged).
cudaError_t launch_group_runs(const SegDesc* segs, uint32_t n_segs, const uint64_t* const* known, cudaStream_t stream);
cudaError_t launch_sort_stage(const SegDesc* segs, uint32_t n_segs, uint32_t n_slots, uint32_t* seg_flags,
                              SortCtl* ctl, SegDesc* resweep_segs, uint64_t* resweep_start, uint64_t* resweep_rend,
                              int grid_tiles, int grid_segs, uint32_t* gstatus, int64_t wait_limit,
                              cudaStream_t stream);
int sort_tile_records();

// Fused merge-sweep (fms.cu): set-up once per process before any launch
// (kernel attribute and grid; not during a stream capture), the launch
// sequence (plan, samples, splitters, merge-sweep), and the table sizes
// for a segment of n records.
cudaError_t fms_prepare(int num_sms);
cudaError_t launch_fms(const SegDesc* segs, SortCtl* ctl, uint32_t* seg_flags, uint32_t* gstatus, int64_t wait_limit,
                       int grid_samples, cudaStream_t stream);
uint64_t fms_max_samples(uint64_t n);
uint64_t fms_max_chunks(uint64_t n);
uint64_t fms_max_super(uint64_t n);

// Message returned by talp_gpu_last_error() on this thread.
void set_last_error(const std::string& msg);

}  // namespace talp
