"""Build step of the CUDA library: nvcc for sm_103a, in-tree shared object."""
from __future__ import annotations

import glob
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
LIB = os.path.join(_HERE, "libgm.so")
SOURCES = [os.path.join(_HERE, "csrc", "gm_lib.cu")]
DEPS = glob.glob(os.path.join(_HERE, "csrc", "*")) + [os.path.join(_ROOT, "include", "gm.h")]

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def build_lib(force: bool = False, verbose: bool = False) -> str:
    """Compile libgm.so for sm_103a unless it is newer than every source."""
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) <= t for p in DEPS + SOURCES):
            return LIB
    cmd = [nvcc()] + NVCC_FLAGS + ["-o", LIB] + SOURCES
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    build_lib(force=True, verbose=True)
