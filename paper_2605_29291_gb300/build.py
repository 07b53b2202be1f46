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
# the checked build: kernels verify their block indices and launch shapes
# (RAPDB_CHECKED) and report a failed check instead of touching memory
LIB_CHECKED = os.path.join(HERE, "librapdb_checked.so")
SOURCES = ["rapdb.cu", "kern_f32.cu", "kern_bf16.cu", "kern_fp8.cu", "rapdb_noalloc.cu", "rapdb_selftest.cu"]
DEPS = SOURCES + ["rapdb_device.cuh", "rapdb_kernels.cuh", "rapdb_sym.cuh", "rapdb_tc.cuh", "rapdb_util.cuh", "rapdb_launch.h",
                  "kern_impl.cuh"]
BUILD_DIR = os.path.join(HERE, "_build")
BUILD_DIR_CHECKED = os.path.join(HERE, "_build_checked")
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


def build(force: bool = False, verbose: bool = False, extra: list | None = None, checked: bool = False) -> str:
    """Compile the translation units in parallel, then link the shared library
    (librapdb_checked.so with checked=True)."""
    lib = LIB_CHECKED if checked else LIB
    bdir = BUILD_DIR_CHECKED if checked else BUILD_DIR
    if not force and not needs_build(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    common = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
              *(["-DRAPDB_CHECKED"] if checked else []), *(extra or [])]
    procs, objs = [], []
    for f in SOURCES:
        obj = os.path.join(bdir, f.replace(".cu", ".o"))
        objs.append(obj)
        cmd = common + ["-c", os.path.join(CSRC, f), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((f, subprocess.Popen(cmd)))
    failed = [f for f, pr in procs if pr.wait() != 0]
    if failed:
        raise RuntimeError(f"nvcc failed on {failed}")
    link = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", lib + ".tmp", *objs]
    if verbose:
        print(" ".join(link), flush=True)
    subprocess.run(link, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None, checked="--checked" in sys.argv)
