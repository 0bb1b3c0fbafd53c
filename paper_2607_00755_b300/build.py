"""Build libkx.so in-tree for sm_103a (B300) with nvcc, and the bounds-checked
libkx_check.so (the same sources with -DKX_CHECK).

Usage: python -m paper_2607_00755_b300.build [--force] [--check]
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkx.so")
OBJ_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libkx_check.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler",
          "-ffp-contract=off", f"-I{INCLUDE}"]
# The kernel-tensor build is compiled without FMA contraction so that its
# support and Theta decisions are the IEEE results of the written expressions.
PER_FILE = {"kx_build.cu": ["-fmad=false"]}
SOURCES = ["kx_build.cu", "kx_contract.cu", "kx_batch.cu", "kx_api.cu", "kx_serve.cu", "kx_noalloc.cu",
           "kx_sources.cu"]
HEADERS = ["kx_internal.cuh", "kx_math.cuh", "kx_lean.cuh", "kx_ptx.cuh", os.path.join(INCLUDE, "kx.h")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or cand == "nvcc"):
            return cand
    return "nvcc"


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Compile the sources that are out of date (in parallel) and link the
    library; check = True builds libkx_check.so with -DKX_CHECK."""
    obj_dir, lib = (OBJ_CHECK, LIB_CHECK) if check else (OBJ, LIB)
    extra = ["-DKX_CHECK"] if check else []
    os.makedirs(obj_dir, exist_ok=True)
    hdrs = [h if os.path.isabs(h) else os.path.join(CSRC, h) for h in HEADERS]
    objs, procs = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _newer(obj, [path] + hdrs):
            cmd = [nvcc(), *ARCH, *COMMON, *extra, *PER_FILE.get(src, []), "-c", path, "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((subprocess.Popen(cmd), cmd))
    failed = [cmd for p, cmd in procs if p.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, failed[0])
    if force or _newer(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, check="--check" in sys.argv)
