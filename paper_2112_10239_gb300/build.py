"""Build ``libtlq.so`` (the CUDA library behind the C-ABI in ``include/tlq.h``).

One ``nvcc`` per translation unit, run in parallel, for sm_103a only, then one link
step. The library lands next to this file (in-tree, git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtlq.so")
INCLUDE = os.path.join(ROOT, "include")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
          "-I", INCLUDE, "-I", CSRC]
SOURCES = ["cone.cu", "cone_global.cu", "dense.cu", "density.cu", "tiny.cu", "mps.cu", "noalloc.cu", "api.cpp",
           "planner.cpp", "serving.cpp"]
HEADERS = ["internal.h", "runtime.h", "gates.cuh", "tc.cuh"]
# Per-source flags, each measured against ptxas -O3 on the same GPU: the cone kernel's
# shared-memory tier (cone.cu) at -O1 (the n=500 batch 4.01 -> 3.90 ms, the n=20 batch
# level), its global-memory tier (cone_global.cu, which includes cone.cu) at -O3 (-O1 was
# 10 % slower there), the dense passes (dense.cu) at -O1 (n=28 energy 0.569 -> 0.579 of
# HBM, energy + gradient 0.585 -> 0.605) and the MPS route (mps.cu) at -O1 (the n=20 batch
# 30.4 -> 27.7 ms, n=500 level). The partial trace (density.cu) stays at -O3 (-O1: 1 % slower).
SOURCE_FLAGS = {"cone.cu": ["-Xptxas", "-O1"], "dense.cu": ["-Xptxas", "-O1"], "mps.cu": ["-Xptxas", "-O1"]}
SOURCE_DEPS = {"cone_global.cu": ["cone.cu"]}


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.exists(d) and os.path.getmtime(d) > t for d in deps)


def _compile(src, extra):
    path = os.path.join(CSRC, src)
    obj = os.path.join(OBJ, src + ".o")
    deps = [path, os.path.join(INCLUDE, "tlq.h"), os.path.abspath(__file__)] + \
        [os.path.join(CSRC, h) for h in HEADERS + SOURCE_DEPS.get(src, [])]
    if not _stale(obj, deps):
        return obj, ""
    lang = ["-x", "cu"] if src.endswith(".cu") else ["-x", "c++"]
    cmd = [NVCC] + ARCH + COMMON + SOURCE_FLAGS.get(src, []) + extra + lang + ["-c", path, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj, r.stderr


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(OBJ, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra)), srcs))
    objs = [o for o, _ in results]
    if verbose:
        for (o, log) in results:
            if log:
                print(o, log, file=sys.stderr)
    if _stale(LIB, objs):
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(verbose=v or bool(extra), extra=extra))
