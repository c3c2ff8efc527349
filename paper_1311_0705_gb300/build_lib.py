"""Compile the library (CUDA for sm_103a + host C++) into ``_build/libhgrt.so``.

Translation units compile in parallel; the path-calculation units are
built with ``-fmad=false`` (and the host units with ``-ffp-contract=off``) so
that every FP64 multiply and add is rounded on its own, as the arithmetic
contract of the C ABI states.
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhgrt.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# (source, needs -fmad=false)
UNITS = [
    ("trace.cu", True),
    ("batch.cu", True),
    ("noalloc.cu", True),
    ("gbuild.cu", True),
    ("metrics.cu", False),
    ("grid.cpp", False),
    ("build.cpp", False),
    ("common.cpp", False),
]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhgrt")


def _cuda_home(nvcc: str) -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "hgrt.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def _compile(args):
    src, nofma, nvcc, verbose = args
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, src + ".o")
    inc = ["-I", INCLUDE, "-I", CSRC]
    if src.endswith(".cu"):
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
               "--expt-relaxed-constexpr", *inc, "-c", path, "-o", obj]
        if nofma:
            cmd.insert(1, "-fmad=false")
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-Wall",
               "-I", os.path.join(_cuda_home(nvcc), "include"), *inc, "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, jobs: int = 0) -> str:
    """Build libhgrt.so if a source changed (or ``force``); return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = jobs or min(len(UNITS), os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(jobs) as ex:
        res = list(ex.map(_compile, [(s, f, nvcc, verbose) for s, f in UNITS]))
    if verbose:
        for obj, err in res:
            if err.strip():
                sys.stderr.write(err)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *[o for o, _ in res], "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
