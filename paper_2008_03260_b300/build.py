"""Compile the CUDA library ``libslash.so`` in place (sm_103a only), and its
checked twin ``libslash_checked.so`` (-DSLASH_CHECKS: data-derived indices are
tested before use; see slash_debug_bounds in include/slash.h).

Usage: ``python -m paper_2008_03260_b300.build [--force] [--checked]``.  nvcc
cross-compiles without a GPU, so this runs on a CPU-only machine too.
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libslash.so")
LIB_CHECKED = os.path.join(PKG, "libslash_checked.so")
SOURCES = [os.path.join(CSRC, "slash.cu"), os.path.join(CSRC, "slash_topkapi.cu"),
           os.path.join(CSRC, "slash_probe.cu"), os.path.join(CSRC, "slash_serve.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [
    os.path.join(INCLUDE, "slash.h"), os.path.join(INCLUDE, "slash_topkapi.h"), os.path.join(INCLUDE, "slash_serve.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-shared", "-I", INCLUDE, "-I", CSRC]


def needs_build(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in DEPS if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if force or needs_build(checked):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC, *FLAGS, *(["-DSLASH_CHECKS"] if checked else []), "-o", tmp, *SOURCES]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
