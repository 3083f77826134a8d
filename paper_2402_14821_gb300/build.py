"""Builds the CUDA library libbp_lb.so in-tree with nvcc for sm_103a (GB300)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libbp_lb.so")
SOURCES = ("bp_lb.cu", "bp_lb_inst_ragged_i32.cu", "bp_lb_inst_ragged_i64.cu",
           "bp_lb_inst_nodes.cu", "bp_lb_noalloc.cu", "bp_serve.cu", "bp_lb_probe.cu")
DEPS = SOURCES + ("bp_lb_core.cuh", "bp_lb_eval.cuh", "bp_lb_kernels.cuh", "bp_lb_launch.cuh",
                  "bp_lb_prefix.cuh", "bp_lb_vb2.cuh", "bp_lb_l2.cuh", "bp_lb_cluster.cuh")
ARCH = ("-gencode", "arch=compute_103a,code=sm_103a")


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    srcs = [os.path.join(CSRC, d) for d in DEPS]
    srcs.append(os.path.join(HERE, "..", "include", "bp_lb.h"))
    return any(os.path.getmtime(s) > t for s in srcs if os.path.exists(s))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libbp_lb.so (no-op when it is newer than every source).  The
    translation units compile in parallel, then link into one shared library."""
    if not force and not _stale(LIB):
        return LIB
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]
    if verbose:
        flags.append("-Xptxas=-v")
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        objs.append(obj)
        procs.append((src, subprocess.Popen(["nvcc", *flags, "-c", os.path.join(CSRC, src),
                                              "-o", obj])))
    failed = [src for src, p in procs if p.wait() != 0]
    if failed:
        raise RuntimeError(f"nvcc failed on {failed}")
    subprocess.run(["nvcc", *ARCH, "-shared", "-o", LIB + ".tmp", *objs], check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
