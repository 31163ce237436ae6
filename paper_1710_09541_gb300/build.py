"""Compile the CUDA library in-tree with nvcc for sm_103a (GB300).

    python -m paper_1710_09541_gb300.build

writes ``paper_1710_09541_gb300/_lib/liblbm_pf.so``.  The CUDA runtime is
linked statically, so the library needs only the NVIDIA driver at run time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc", "lbm_pf.cu")
DEPS = [SRC, os.path.join(PKG, "csrc", "lbm_kernels.cuh"), os.path.join(PKG, "csrc", "lbm_store.cuh"),
        os.path.join(ROOT, "include", "lbm_pf.h")]
LIB_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIB_DIR, "liblbm_pf.so")
# the same library with the step's index checks and halo poisoning compiled in
LIB_DEBUG = os.path.join(LIB_DIR, "liblbm_pf_debug.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm_pf.so")


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build the release library (or, with debug=True, the checking one)."""
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(lib):
        return lib
    os.makedirs(LIB_DIR, exist_ok=True)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-o", tmp, SRC]
    if debug:
        cmd.insert(1, "-DLBM_DEBUG_CHECKS=1")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
