"""Build libdeam.so in-tree with nvcc for sm_103a (no cmake, two translation
units compiled in parallel, one -gencode)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdeam.so")
# the bounds-checked build (-DDEAM_BOUNDS_CHECK): guarded device accesses record
# an out-of-range index and the entry point returns DEAM_ERR_ARG
LIB_CHECKED = os.path.join(HERE, "libdeam_checked.so")
SOURCES = ["deam_kernels.cu", "deam_backproject.cu", "deam_api.cu", "deam_batch.cu", "deam_noalloc.cu", "deam_mar.cu"]
HEADERS = ["deam_internal.h", "deam_epilogue.cuh", "deam_ctx.h", os.path.join("..", "..", "include", "deam.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdeam.so")


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, h) for h in HEADERS]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, bounds_check: bool = False) -> str:
    """Compile (if needed) and return the path of libdeam.so, or with
    bounds_check=True of the bounds-checked libdeam_checked.so."""
    lib = LIB_CHECKED if bounds_check else LIB
    out_dir = OUT_DIR + ("_checked" if bounds_check else "")
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [cc, *ARCH, *FLAGS, *(["-DDEAM_BOUNDS_CHECK"] if bounds_check else []), "-c",
               os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{out.decode(errors='replace')}")
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, bounds_check="--bounds-check" in sys.argv))
