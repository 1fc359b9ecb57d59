// Internal hooks of the context used by the serving loop and the raw
// adapter (not part of the C ABI).
#pragma once
#include <cstdint>

#include "../../include/talp_gpu.h"
#include "common.cuh"

namespace talp {

// Device descriptor of a trace for the finalize kernel, its number of
// regions, or nullptr when the trace is unknown.
const TraceDev* trace_device_desc(talp_gpu_ctx* c, uint64_t trace_id, uint32_t* n_regions);

// The context's device index.
int ctx_device(talp_gpu_ctx* c);

// Count a server as a user of the context (destroy refuses while any exist).
void ctx_hold(talp_gpu_ctx* c, int delta);

// Drop the held-back raw records of a trace (TALP_GPU_ALL: of every trace).
void raw_hold_drop(talp_gpu_ctx* c, uint64_t trace_id);

// Raw records of a trace currently held back.
uint64_t raw_held_records(talp_gpu_ctx* c, uint64_t trace_id);

}  // namespace talp
