"""Build the CUDA library in-tree for sm_103a (B300).

    python -m paper_2603_26576_b300.build [--force]

Produces paper_2603_26576_b300/libtalp_gpu.so from csrc/*.cu with nvcc.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libtalp_gpu.so")
SOURCES = ["sweep.cu", "reduce.cu", "sort.cu", "fms.cu", "capi.cu", "noalloc.cu", "serve.cu", "concurrency.cu", "raw.cu"]
HEADERS = ["common.cuh", "sweep_core.cuh", "kernels.h", "engine.h"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "--fmad=false",
    "-Xcompiler", "-fPIC,-O2,-ffp-contract=off",
    "-cudart=shared",
    "-I", os.path.join(ROOT, "include"),
]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "talp_gpu.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force=False, verbose=False, extra_flags=()):
    if not force and not _stale():
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC, *NVCC_FLAGS, *extra_flags, "-shared", "-o", tmp,
           *[os.path.join(CSRC, f) for f in SOURCES],
           "-Xlinker", f"-rpath,{CUDA_HOME}/lib64"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra_flags=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else [])
    print(LIB)
