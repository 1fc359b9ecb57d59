"""B300 reducer of host/device traces into the extended POP efficiency metrics.

Thin Python binding over the C ABI in include/talp_gpu.h (libtalp_gpu.so,
built in-tree for sm_103a).  Every step of the computation runs in the CUDA
library; this module only marshals arguments.  There is no CPU fallback: if
the library is missing, importing the binding's functions raises.
"""
from ._lib import (  # noqa: F401
    TALP_GPU_ALL, TALP_GPU_ALL_REGIONS, TALP_GPU_APPEND, TALP_GPU_HOLD_BACK, TALP_GPU_NOT_SORTED, TALP_GPU_GROUPED_BY_STREAM, TALP_GPU_DEVICE_PTRS, TALP_GPU_MAX_REGIONS,
    TALP_GPU_SORTED_BY_START, TalpGpuError, LIB_PATH, Context, batch_from_arrays, load_library,
    metrics_to_dict, metrics_from_dict, talp_gpu_metrics_combine, talp_gpu_concurrency, TALP_GPU_CONC_LEVELS, talp_gpu_scalability, talp_gpu_ingest_raw, talp_gpu_raw_held,
    raw_batch_from_arrays, talp_gpu_raw_batch, talp_gpu_create, talp_gpu_destroy, talp_gpu_ingest_events, talp_gpu_last_error,
    talp_gpu_memory, talp_gpu_region_metrics, talp_gpu_region_metrics_batch, talp_gpu_region_metrics_device,
    talp_gpu_thread_metrics, talp_gpu_thread_metrics_device, talp_gpu_thread_tree, thread_tree_from_bytes,
    talp_gpu_thread_metrics_combine,
    talp_gpu_reset, talp_gpu_unit_sums, talp_gpu_profile, talp_gpu_profile_read, talp_gpu_reduce_noalloc,
    TALP_GPU_NOALLOC_MAX_UNITS, TALP_GPU_PLAN_AUTOTUNE, Plan, talp_gpu_plan_create, talp_gpu_plan_launch,
    talp_gpu_plan_metrics, talp_gpu_plan_info, talp_gpu_plan_destroy, talp_gpu_metrics, talp_gpu_trace_batch, EXPORTED_SYMBOLS,
    Server, talp_gpu_server_create, talp_gpu_server_open_job, talp_gpu_server_submit, talp_gpu_server_submit_raw, talp_gpu_server_query, talp_gpu_server_query_threads,
    talp_gpu_server_drain, talp_gpu_server_close_job, talp_gpu_server_info, talp_gpu_server_destroy,
)
