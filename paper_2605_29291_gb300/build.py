"""Build the CUDA library librapdb.so in-tree for sm_103a (GB300) with nvcc.

The library is a plain C ABI (include/rapdb.h) over hand-written CUDA; it
links only the CUDA runtime.  `build()` recompiles when a source is newer
than the library.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "librapdb.so")
SOURCES = ["rapdb.cu", "kern_f32.cu", "kern_bf16.cu", "kern_fp8.cu", "rapdb_noalloc.cu", "rapdb_selftest.cu"]
DEPS = SOURCES + ["rapdb_device.cuh", "rapdb_kernels.cuh", "rapdb_util.cuh", "rapdb_launch.h", "kern_impl.cuh"]
BUILD_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return "nvcc"


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in DEPS] + [os.path.join(INCLUDE, "rapdb.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra: list | None = None) -> str:
    """Compile the translation units in parallel, then link the shared library."""
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    common = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
              *(extra or [])]
    procs, objs = [], []
    for f in SOURCES:
        obj = os.path.join(BUILD_DIR, f.replace(".cu", ".o"))
        objs.append(obj)
        cmd = common + ["-c", os.path.join(CSRC, f), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((f, subprocess.Popen(cmd)))
    failed = [f for f, pr in procs if pr.wait() != 0]
    if failed:
        raise RuntimeError(f"nvcc failed on {failed}")
    link = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", LIB + ".tmp", *objs]
    if verbose:
        print(" ".join(link), flush=True)
    subprocess.run(link, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
