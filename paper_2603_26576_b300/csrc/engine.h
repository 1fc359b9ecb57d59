// Internal hooks of the context used by the serving loop (not part of the
// C ABI).
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

}  // namespace talp
