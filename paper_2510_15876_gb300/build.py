"""Build the CUDA library (libafr.so) in-tree for sm_103a, and its debug
build (libafr_debug.so, with AFR_DEBUG: device-side index checks and the test
hooks of include/afr_debug.h).

Each translation unit under csrc/ compiles in parallel with nvcc; the objects
link into paper_2510_15876_gb300/libafr.so and libafr_debug.so. Rebuilds only
when a source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libafr.so")
DEBUG_LIB = os.path.join(PKG, "libafr_debug.so")   # AFR_DEBUG: device checks and the hooks of include/afr_debug.h
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libafr.so")
    return cand


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    return max(os.path.getmtime(d) for d in deps) > os.path.getmtime(lib)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compiles libafr.so and libafr_debug.so (the same sources with
    AFR_DEBUG); every translation unit of both in parallel."""
    targets = [(LIB, "release", []), (DEBUG_LIB, "debug", ["-DAFR_DEBUG"])]
    todo = [t for t in targets if force or _stale(t[0])]
    if not todo:
        return LIB
    nvcc = _nvcc()
    base = NVCC_FLAGS + ARCH + (extra or [])

    def one(job):
        src, odir, defs = job
        obj = os.path.join(odir, os.path.basename(src)[:-3] + ".o")
        r = subprocess.run([nvcc, *base, *defs, "-c", src, "-o", obj], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    jobs = []
    for lib, tag, defs in todo:
        odir = os.path.join(BUILD, tag)
        os.makedirs(odir, exist_ok=True)
        jobs += [(src, odir, defs) for src in sources()]
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(one, jobs))
    for lib, tag, _ in todo:
        mine = [o for o in objs if os.path.dirname(o) == os.path.join(BUILD, tag)]
        tmp = lib + f".{os.getpid()}.tmp"
        r = subprocess.run([nvcc, "-shared", *ARCH, "-o", tmp, *mine, "-lcudart"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
