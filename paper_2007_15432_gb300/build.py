"""Builds ``libp3t.so`` (sm_103a) in-tree with nvcc.

Each CUDA source is compiled to an object in parallel, then linked into a
shared library with the CUDA runtime linked statically.  Sources whose
arithmetic must be bit-identical on every IEEE machine (keys and grid
geometry, the neighbour predicate, the Hermite block steps) are compiled with
``-fmad=false``; the tree walk keeps FMA contraction; the all-pairs kernels
flush FP32 subnormals.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libp3t.so")

SOURCES = ["primitives.cu", "tree.cu", "walk.cu", "neighbours.cu", "hard.cu", "ctx.cu",
           "noalloc.cu", "adjoint.cu", "direct.cu", "hermite_adj.cu"]
NO_FMA = {"tree.cu", "neighbours.cu", "hard.cu", "ctx.cu", "noalloc.cu", "hermite_adj.cu"}
# FP32 subnormals flushed to zero (the all-pairs kernels' FP32 operands are
# far from 2^-126; rsqrtf then needs no subnormal handling)
FTZ = {"direct.cu"}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, "p3t_internal.cuh"), os.path.join(CSRC, "exact_conv.cuh"),
              os.path.join(INCLUDE, "p3t.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles and links libp3t.so unless it is newer than every source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(OBJDIR, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        if src in NO_FMA:
            cmd.insert(len(ARCH) + 1, "-fmad=false")
        if src in FTZ:
            cmd.insert(len(ARCH) + 1, "-ftz=true")
        if verbose:
            cmd.insert(len(ARCH) + 1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            print(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
