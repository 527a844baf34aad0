"""Compile the CUDA library in-tree: paper_2002_11710_gb300/_build/libasched.so.

sm_103a only (GB300); four translation units compiled in parallel and linked into
one shared library, so it builds in under a minute here and on the GPU host alike.
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRCS = [os.path.join(PKG, "csrc", n) for n in ("asched.cu", "sweep.cu", "matrix.cu", "peaks.cu")]
HDR = os.path.join(ROOT, "include", "asched.h")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libasched.so")

# No -use_fast_math (nor -ftz/-prec-* overrides): the travel-matrix screen's error bounds
# rest on the documented accuracy of sinf, asinf and rsqrtf in the default mode.
NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC",
]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(x) for x in SRCS + [HDR, os.path.join(PKG, "csrc", "nvtx_range.h")])
    stale = not os.path.exists(LIB) or os.path.getmtime(LIB) < newest
    if force or stale:
        tag = f".tmp{os.getpid()}"
        inc = ["-I", os.path.join(ROOT, "include")]
        objs, procs = [], []
        try:
            for src in SRCS:
                obj = os.path.join(OUT_DIR, os.path.basename(src) + tag + ".o")  # nvcc reads the suffix
                cmd = [nvcc(), *NVCC_FLAGS, *inc, "-c", "-o", obj, src]
                if verbose:
                    cmd.insert(1, "-Xptxas=-v")
                    print(" ".join(cmd), file=sys.stderr)
                objs.append(obj)
                procs.append(subprocess.Popen(cmd))
            codes = [p.wait() for p in procs]
            if any(codes):
                raise subprocess.CalledProcessError(next(c for c in codes if c), "nvcc")
            tmp = os.path.join(OUT_DIR, "libasched" + tag + ".so")
            subprocess.check_call([nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                                   "-o", tmp, *objs])
            os.replace(tmp, LIB)
        finally:
            for p in procs:
                if p.poll() is None:
                    p.wait()
            for obj in objs:
                if os.path.exists(obj):
                    os.remove(obj)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
