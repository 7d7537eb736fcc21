"""Build step of libeigdc.so: nvcc for sm_103a, in-tree, no cmake.

Compiles the translation units under csrc/ in parallel (one -gencode:
arch=compute_103a, code=sm_103a) and links them into
paper_1011_3077_gb300/libeigdc.so next to this file.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libeigdc.so")
SOURCES = ["linalg.cu", "misc.cu", "leaves.cu", "tc_gemm.cu", "tcx_gemm.cu", "api.cu", "noalloc.cu",
           "cplane.cu", "trevc.cu", "fused.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("command failed: %s\n%s" % (" ".join(cmd), p.stdout))
    return p.stdout


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src, os.path.join(CSRC, "internal.h"), os.path.join(CSRC, "tc_ptx.cuh"),
            os.path.join(CSRC, "cplane_strategy.h"), os.path.join(CSRC, "jacobi_leaf.cuh"),
            os.path.join(CSRC, "fused_dev.cuh"),
            os.path.join(os.path.dirname(HERE), "include", "eigdc.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(verbose=False, force=False):
    """Compile (if stale) and link libeigdc.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, s):
            jobs.append([nvcc] + ARCH + FLAGS + ["-c", s, "-o", o])
    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for out in ex.map(_run, jobs):
                if verbose and out.strip():
                    print(out)
    if force or jobs or not os.path.exists(LIB):
        # --no-undefined: a missing definition fails the link, not the first load
        _run([nvcc] + ARCH + ["-shared", "-Xlinker", "--no-undefined", "-o", LIB] + objs)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
