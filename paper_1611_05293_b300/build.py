"""Build the in-tree CUDA library libvfps.so for sm_103a with nvcc.

The library is the whole compute path: kernels (csrc/vfps_kernels.cuh),
runtime and C ABI (csrc/vfps.cu, include/vfps.h) and the host impedance
tables (csrc/impedance_host.cpp).  The Python binding only loads it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libvfps.so")
LIB_DEBUG = os.path.join(HERE, "libvfps_debug.so")  # -DVFPS_DEBUG: shared-memory index checks
SOURCES = [os.path.join(CSRC, f) for f in ("vfps.cu", "impedance_host.cpp")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".cuh", ".h"))] + \
    [os.path.join(ROOT, "include", "vfps.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in DEPS)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build libvfps.so (or, with debug, libvfps_debug.so: the same code with
    the shared-memory index checks of VFPS_DEBUG compiled in)."""
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(lib):
        return lib
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), "-o", lib + ".tmp", *SOURCES, "-lcudart"]
    if debug:
        cmd.insert(1, "-DVFPS_DEBUG")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
