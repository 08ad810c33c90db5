"""Build the CUDA library in-tree: nvcc for sm_103a, one .so next to this file."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libtachiom.so")
SOURCES = ["index.cu", "search.cu", "k_topc.cu", "k_topc_tc.cu", "k_gather.cu", "k_refine.cu", "profile.cu", "refine_noalloc.cu", "k_refine_tc.cu", "server.cu", "k_topc_tc1.cu", "k_refine_dec.cu", "tac.cu", "tac_cluster.cu", "budgets.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    raise RuntimeError("nvcc not found")


def build(force: bool = False, verbose: bool = False, jobs: int = 8) -> str:
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    hdrs = [os.path.join(CSRC, "tachiom_internal.cuh"), os.path.join(CSRC, "tc_common.cuh"),
            os.path.join(os.path.dirname(HERE), "include", "tachiom.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) <= t for p in srcs + hdrs):
            return LIB
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    common = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
    if verbose:
        common += ["-Xptxas", "-v"]
    procs, objs = [], []
    for s in srcs:
        o = os.path.join(objdir, os.path.basename(s) + ".o")
        objs.append(o)
        procs.append(subprocess.Popen(common + ["-c", s, "-o", o]))
        if len(procs) >= jobs:
            if procs.pop(0).wait() != 0:
                raise RuntimeError("nvcc failed")
    for p in procs:
        if p.wait() != 0:
            raise RuntimeError("nvcc failed")
    tmp = LIB + ".tmp"
    subprocess.check_call([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lcublas"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
