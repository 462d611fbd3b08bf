"""Compile libstiles.so in-tree for sm_103a (nvcc; works without a GPU)."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libstiles.so")
SOURCES = ["capi.cu", "analyze.cpp", "noalloc.cu"]
HEADERS = ["plan.h", "device_common.cuh", "factor_f64.cuh", "factor_lp.cuh", "factor_oz.cuh", "solve.cuh", "aux_kernels.cuh",
           "selinv.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _newest_input():
    paths = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    paths.append(os.path.join(os.path.dirname(PKG), "include", "stiles.h"))
    return max(os.path.getmtime(p) for p in paths if os.path.exists(p))


def build_library(force=False, verbose=False):
    """Build (or reuse an up-to-date) libstiles.so; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, "-shared", "-Xcompiler", "-fPIC", "-O3", "-std=c++17", "-lineinfo", *ARCH,
           "-o", LIB + ".tmp", *[os.path.join(CSRC, s) for s in SOURCES]]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError(f"nvcc failed ({res.returncode}) building {LIB}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose="-v" in sys.argv))
