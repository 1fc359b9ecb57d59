"""CPU-only checks of the C-ABI library: it loads, exports every function the
header declares, and the binding's structs match the header's layout.  No
compute call is made (there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "talp_gpu.h")


def _declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(talp_gpu_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    fns = _declared_functions()
    for f in ("talp_gpu_create", "talp_gpu_destroy", "talp_gpu_ingest_events", "talp_gpu_region_metrics",
              "talp_gpu_reset"):
        assert f in fns


def test_library_exports_every_declared_symbol():
    import paper_2603_26576_b300 as P
    lib = P.load_library()
    for f in _declared_functions():
        assert hasattr(lib, f), f
    assert set(_declared_functions()) == set(P.EXPORTED_SYMBOLS)


def test_struct_layouts_match_header():
    import paper_2603_26576_b300 as P
    # talp_gpu_trace_batch: 8 + 4*4 + 8 pointers; talp_gpu_metrics: 8 + 4*4 + 11*8 + 9*8
    assert ctypes.sizeof(P.talp_gpu_trace_batch) == 8 + 16 + 8 * 8
    assert ctypes.sizeof(P.talp_gpu_metrics) == 8 + 16 + 11 * 8 + 9 * 8
    hdr = open(HEADER).read()
    body = hdr[hdr.index("typedef struct {\n    uint64_t trace_id;\n    uint32_t region;"):]
    body = body[:body.index("} talp_gpu_metrics;")]
    fields = re.findall(r"\b(?:uint64_t|uint32_t|int64_t|double)\s+(\w+);", body)
    assert fields == [f for f, _ in P.talp_gpu_metrics._fields_]


def test_errors_without_a_gpu_are_clean():
    import torch
    import paper_2603_26576_b300 as P
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.TalpGpuError) as ei:
        P.talp_gpu_create(0)
    assert ei.value.status in (-1, -3)
    # a null context is refused without touching CUDA
    lib = P.load_library()
    assert lib.talp_gpu_reset(None, 0) == -1
    assert lib.talp_gpu_destroy(None) == 0
    assert "null" in P.talp_gpu_last_error()
