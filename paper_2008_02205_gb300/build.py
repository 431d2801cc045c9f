"""Build the CUDA library (libmlpg.so) in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into one shared
library next to this file.  Host code is compiled without floating-point
contraction so that host geometry rounds the same way on x86 and Arm.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(HERE, "libmlpg.so")
SOURCES = ["api.cu", "neighbors.cu", "assemble.cu", "assemble3d.cu", "cells2d.cu", "operators.cu", "krylov.cu", "noalloc.cu", "geometry.cpp",
           "quadrature.cpp", "tiles.cpp", "cells3d.cu"]
# per-file flags: the device 3D cell builder rounds like the host builder (no contraction)
EXTRA = {"cells3d.cu": ["--fmad=false"]}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    raise RuntimeError("nvcc not found")


def _flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC] + ARCH


def _compile(src):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    path = os.path.join(CSRC, src)
    deps = [path, os.path.join(CSRC, "internal.h"), os.path.join(ROOT, "include", "mlpg.h")]
    if os.path.exists(obj) and all(os.path.getmtime(obj) >= os.path.getmtime(d) for d in deps):
        return obj
    lang = ["-x", "cu"] if src.endswith(".cu") else []
    cmd = [nvcc()] + _flags() + EXTRA.get(src, []) + lang + ["-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    if not os.path.exists(SO) or any(os.path.getmtime(o) > os.path.getmtime(SO) for o in objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", SO] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    if verbose:
        print(SO)
    return SO


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
