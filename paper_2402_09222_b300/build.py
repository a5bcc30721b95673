"""Build libmcx.so in-tree with nvcc for sm_103a (B300).

Translation units that evaluate the plain definition's FP64 arithmetic
(transport, exact lookup, adjoint) are compiled with --fmad=false so that no
multiply-add is fused; the fast lookup and the host layer use the defaults.
--bounds builds the bounds-checked debug library libmcx_bounds.so instead
(MCX_BOUNDS_CHECK=1; loaded by the binding when MCX_LIB=bounds).
Usage:  python -m paper_2402_09222_b300.build [--force] [--verbose-ptxas] [--bounds]
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libmcx.so")
LIB_BOUNDS = os.path.join(HERE, "libmcx_bounds.so")
BUILD = os.path.join(ROOT, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
EXACT_TUS = {"transport.cu", "xs_exact.cu", "adjoint.cu"}
SOURCES = ["mcx_api.cu", "xs_exact.cu", "xs_fast.cu", "transport.cu", "adjoint.cu", "noalloc.cu",
           "eigen.cu"]
HEADERS = ["mcx_internal.cuh", "xs_exact.cuh", "kernels.h"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, ptxas_verbose: bool = False, bounds: bool = False) -> str:
    out_dir = os.path.join(BUILD, "bounds") if bounds else BUILD
    lib = LIB_BOUNDS if bounds else LIB
    os.makedirs(out_dir, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "mcx.h")]
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [path] + headers):
            cmd = [nvcc()] + ARCH + COMMON + ["-c", path, "-o", obj]
            if bounds:
                cmd.append("-DMCX_BOUNDS_CHECK=1")
            if src in EXACT_TUS:
                cmd.append("--fmad=false")
            if ptxas_verbose:
                cmd += ["-Xptxas", "-v"]
            subprocess.check_call(cmd)
    if force or _stale(lib, objs):
        subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", lib] + objs)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, ptxas_verbose="--verbose-ptxas" in sys.argv,
                bounds="--bounds" in sys.argv))
