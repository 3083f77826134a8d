"""Builds the CUDA library libbp_lb.so in-tree with nvcc for sm_103a (GB300)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libbp_lb.so")
SOURCES = ("bp_lb.cu",)
DEPS = ("bp_lb.cu", "bp_lb_core.cuh", "bp_lb_eval.cuh", "bp_lb_kernels.cuh")
ARCH = ("-gencode", "arch=compute_103a,code=sm_103a")


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    srcs = [os.path.join(CSRC, d) for d in DEPS]
    srcs.append(os.path.join(HERE, "..", "include", "bp_lb.h"))
    return any(os.path.getmtime(s) > t for s in srcs if os.path.exists(s))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libbp_lb.so (no-op when it is newer than every source)."""
    if not force and not _stale(LIB):
        return LIB
    cmd = ["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-o", LIB + ".tmp", *[os.path.join(CSRC, s) for s in SOURCES]]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
