"""Build step of the CUDA library: nvcc for sm_103a, in-tree shared object.

The host code and each list of kernel template instances are separate
translation units (csrc/gm_lib.cu, csrc/gm_inst_*.cu), compiled in parallel
to objects under _build/ and linked into libgm.so."""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
LIB = os.path.join(_HERE, "libgm.so")
BUILD_DIR = os.path.join(_HERE, "_build")
SOURCES = sorted(glob.glob(os.path.join(_HERE, "csrc", "*.cu")))
HEADERS = sorted(glob.glob(os.path.join(_HERE, "csrc", "*.cuh")) + glob.glob(os.path.join(_HERE, "csrc", "*.h")) +
                 [os.path.join(_ROOT, "include", "gm.h")])

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     # kernel template instances are launched from another translation unit
                     "-static-global-template-stub=false"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _obj(src: str) -> str:
    return os.path.join(BUILD_DIR, os.path.splitext(os.path.basename(src))[0] + ".o")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(p) > t for p in deps)


def build_lib(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile libgm.so for sm_103a unless it is newer than every source and header."""
    if not force and not _stale(LIB, SOURCES + HEADERS):
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    todo = [s for s in SOURCES if force or _stale(_obj(s), [s] + HEADERS)]

    def compile_one(src):
        cmd = [nvcc()] + NVCC_FLAGS + ["-c", src, "-o", _obj(src)]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r

    with ThreadPoolExecutor(max_workers=jobs or min(len(todo) or 1, os.cpu_count() or 1)) as ex:
        results = list(ex.map(compile_one, todo))
    for src, r in results:
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}{r.stderr}")
    cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB] + [_obj(s) for s in SOURCES]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    build_lib(force=True, verbose=True)
