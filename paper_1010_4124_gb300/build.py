"""Build libklb.so (the C-ABI library, CUDA for sm_103a) in-tree.

nvcc compiles each translation unit in parallel for exactly one target,
`-gencode arch=compute_103a,code=sm_103a`, with `-lineinfo`, and links a
shared library next to this file.  No cmake; a rebuild is skipped when the
library is newer than every source.

build(checked=True) builds the debug variant libklb_checked.so with
-DKLB_CHECK_BOUNDS: every global index of the kernels is checked against
its buffer, an index out of range is skipped and reported by klb_sync
(KLB_E_BOUNDS), nothing traps.
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libklb.so")
LIB_CHECKED = os.path.join(HERE, "libklb_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
              "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(ROOT, "include", "klb.h")]
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list | None = None, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(BUILD, exist_ok=True)
    # processes that start together (ranks of one job) build one at a time;
    # the later ones find the library up to date
    with open(os.path.join(BUILD, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if not force and not _stale(lib):
            return lib
        flags = (extra or []) + (["-DKLB_CHECK_BOUNDS"] if checked else [])
        return _build_locked(verbose, flags, lib, os.path.join(BUILD, "checked") if checked else BUILD)


def _build_locked(verbose: bool, extra: list, lib: str, objdir: str) -> str:
    nvcc = _nvcc()
    os.makedirs(objdir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        # FP64 parity translation units round every multiply and add separately
        per_file = ["-fmad=false"] if src.endswith("_f64.cu") else []
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *per_file, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None, checked="--checked" in sys.argv)
