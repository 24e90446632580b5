"""Compiles the solver's CUDA sources into the in-tree shared library libpdlp_b300.so
(sm_103a only).  Run as a script or call build()."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", f) for f in ("pdlp.cu", "layout.cpp", "noalloc.cu", "mlp.cu")]
DEPS = [os.path.join(HERE, "csrc", f) for f in sorted(os.listdir(os.path.join(HERE, "csrc")))
        if f.endswith((".cu", ".cuh", ".h", ".cpp"))] + [os.path.join(ROOT, "include", "pdlp.h"), __file__]
LIB = os.path.join(HERE, "libpdlp_b300.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include")]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in DEPS)


CEIL_SRC = os.path.join(HERE, "csrc", "gather_ceiling.cu")
CEIL_BIN = os.path.join(HERE, "gather_ceiling")


def build_ceiling(force: bool = False) -> str:
    """The gather/stream throughput microbenchmark used by bench.py for the roofline."""
    if force or not os.path.exists(CEIL_BIN) or os.path.getmtime(CEIL_BIN) < os.path.getmtime(CEIL_SRC):
        tmp = CEIL_BIN + f".tmp{os.getpid()}"
        subprocess.check_call([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
                               "-o", tmp, CEIL_SRC])
        os.replace(tmp, CEIL_BIN)
    return CEIL_BIN


PEAK_SRC = os.path.join(HERE, "csrc", "fp64_peak.cu")
PEAK_BIN = os.path.join(HERE, "fp64_peak")


def build_fp64_peak(force: bool = False) -> str:
    """The FP64 fused multiply-add throughput microbenchmark used by bench.py for the
    arithmetic roof of the FP64 kernels."""
    if force or not os.path.exists(PEAK_BIN) or os.path.getmtime(PEAK_BIN) < os.path.getmtime(PEAK_SRC):
        tmp = PEAK_BIN + f".tmp{os.getpid()}"
        subprocess.check_call([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
                               "-o", tmp, PEAK_SRC])
        os.replace(tmp, PEAK_BIN)
    return PEAK_BIN


def build(force: bool = False, verbose: bool = False) -> str:
    build_ceiling(force)
    build_fp64_peak(force)
    if force or stale():
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [NVCC, *FLAGS, "-o", tmp, *SRC]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
