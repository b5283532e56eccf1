"""Build the CUDA library ``libslh.so`` in-tree (``paper_2404_02950_gb300/lib``).

nvcc compiles every translation unit for sm_103a in parallel and links a
shared library with the CUDA runtime linked statically, so the library
depends only on the driver.  Run ``python -m paper_2404_02950_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "lib")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libslh.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_SRCS = ["api.cu", "stage.cu", "stage_rkn.cu", "stage_diag.cu", "gw.cu", "ghost.cu", "tee.cu", "spectrum.cu", "ko.cu", "diag.cu", "noalloc.cu", "alu_rate.cu"]
CXX_SRCS = ["regrid.cpp", "regrid_policy.cpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build step failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(verbose: bool = False, extra_flags=None) -> str:
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(BUILD_DIR, exist_ok=True)
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-I", CSRC, "-Xcompiler", "-fPIC"]
    if extra_flags:
        common += list(extra_flags)
    jobs = []
    for s in CUDA_SRCS:
        obj = os.path.join(BUILD_DIR, s + ".o")
        jobs.append([nvcc, *ARCH, "-lineinfo", *common, "-c", os.path.join(CSRC, s), "-o", obj])
    for s in CXX_SRCS:
        obj = os.path.join(BUILD_DIR, s + ".o")
        jobs.append([nvcc, *common, "-x", "c++", "-c", os.path.join(CSRC, s), "-o", obj])
    logs = []
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        for out in ex.map(_run, jobs):
            logs.append(out)
    objs = [j[-1] for j in jobs]
    tmp = LIB + ".tmp"
    logs.append(_run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-ldl"]))
    os.replace(tmp, LIB)
    if verbose:
        print("\n".join(l for l in logs if l.strip()))
    return LIB


if __name__ == "__main__":
    flags = sys.argv[1:]
    print(build(verbose=True, extra_flags=flags))
