"""Build libst.so (the sm_103a library behind include/st.h) in-tree.

Compiles every translation unit in parallel with nvcc (CUDA) / g++ (host
C++), then links a shared library with a static CUDA runtime.  Output:
paper_2006_12883_gb300/_build/libst.so.  Rebuilds only when a source is newer
than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libst.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["k_fine.cu", "k_fine_tile.cu", "k_level.cu", "k_level4.cu", "k_coarse.cu", "k_krylov.cu", "k_tma.cu", "st_api.cu",
              "st_noalloc.cu", "st_checkpoint.cu",
              "k_sweep2.cu", "k_linres_restrict.cu"]
CPP_SOURCES = ["st_setup.cpp"]
HEADERS = ["st_internal.cuh", "st_kernels.cuh", "st_setup.h"]


def _sources():
    return [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES + HEADERS] + [
        os.path.join(INCLUDE, "st.h"), os.path.abspath(__file__)]


def _up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libst.so; returns its path."""
    if not force and _up_to_date():
        return LIB
    if not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    os.makedirs(BUILD, exist_ok=True)
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-I", CSRC]
    jobs = []
    objs = []
    for f in CU_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append([NVCC] + ARCH + common + ["-lineinfo", "-Xcompiler", "-fPIC", "-c",
                                              os.path.join(CSRC, f), "-o", o])
    cxx = shutil.which("g++") or "g++"
    for f in CPP_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append([cxx, "-O2", "-std=c++17", "-fPIC", "-I", os.path.join(CUDA_HOME, "include"),
                     "-I", INCLUDE, "-c", os.path.join(CSRC, f), "-o", o])
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = LIB + ".tmp"
    _run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
