"""Builds the package's native libraries in-tree.

* ``libkadabra.so`` -- the CUDA kernels and the C ABI (``csrc/kadabra.cu``),
  compiled for sm_103a only, FP contraction off on both device and host
  (the stop test's FP64 expression tree is part of the specification).
* ``libgraphgen.so`` -- the seeded input generators (``csrc/graphgen.cpp``).
"""

from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CU_SRC = os.path.join(HERE, "csrc", "kadabra.cu")
CU_LIB = os.path.join(HERE, "libkadabra.so")
HEADER = os.path.join(ROOT, "include", "kadabra.h")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-lineinfo", "-O3", "--fmad=false", "-std=c++17",
    "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math",
    "-shared",
]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkadabra.so")
    return exe


def _stale(lib: str, *srcs: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in srcs)


def build_kadabra(force: bool = False, extra=()) -> str:
    if force or _stale(CU_LIB, CU_SRC, HEADER):
        tmp = CU_LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *NVCC_FLAGS, *extra, CU_SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, CU_LIB)
    return CU_LIB


CU_LIB_CHECKED = os.path.join(HERE, "libkadabra_checked.so")


def build_checked(force: bool = False) -> str:
    """The same library with KADABRA_CHECKED: every list, frontier-array,
    level-bound, adjacency and hit-counter index of the sampler is checked
    (tests only; the checks record the failing site and fail the sample)."""
    if force or _stale(CU_LIB_CHECKED, CU_SRC, HEADER):
        tmp = CU_LIB_CHECKED + f".tmp{os.getpid()}"
        cmd = [nvcc(), *NVCC_FLAGS, "-DKADABRA_CHECKED", CU_SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, CU_LIB_CHECKED)
    return CU_LIB_CHECKED


def build_all(force: bool = False) -> None:
    from . import graphgen
    with ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build_kadabra, force), ex.submit(graphgen.build, force)]
        for f in futs:
            f.result()
