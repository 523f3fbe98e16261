"""Compile the C-ABI library ``libskel.so`` in-tree for sm_103a.

Host C++ (tree, interpolative decompositions, layout, C-ABI) is compiled with
g++ and OpenMP; the CUDA kernels with nvcc for ``sm_103a`` only. Translation
units are compiled in parallel and linked against the CUDA runtime. The
result lands in ``paper_2310_16668_gb300/_build/libskel.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libskel.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CXX_SOURCES = ["tree.cpp", "skeletonize.cpp", "layout.cpp", "capi.cpp"]
CU_SOURCES = ["apply.cu", "noalloc.cu", "build_gpu.cu"]
# integer cell coordinates must be computed with plain IEEE operations
NO_CONTRACT = {"tree.cpp", "capi.cpp"}


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def _headers():
    out = [os.path.join(INCLUDE, "skel.h")]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return out


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + _headers() + [__file__])


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    cuda = _cuda_home()
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I" + os.path.join(cuda, "include"), "-I" + INCLUDE, "-I" + CSRC]
    jobs = []
    objs = []
    for f in CXX_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if force or _stale(obj, src):
            flags = ["-O3", "-std=c++17", "-fPIC", "-fopenmp", "-Wall", "-Wno-unknown-pragmas"]
            if f in NO_CONTRACT:
                flags.append("-ffp-contract=off")
            jobs.append(["g++", *flags, *inc, "-c", src, "-o", obj])
    for f in CU_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if force or _stale(obj, src):
            jobs.append([os.path.join(cuda, "bin", "nvcc"), *ARCH, "-O3", "-lineinfo", "-std=c++17",
                         "-Xcompiler", "-fPIC", "-Xptxas", "-v" if verbose else "-O3", *inc,
                         "-c", src, "-o", obj])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
            for out in ex.map(_run, jobs):
                if verbose and out:
                    print(out, file=sys.stderr)
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        _run(["g++", "-shared", "-fopenmp", "-o", tmp, *objs,
              "-L" + os.path.join(cuda, "lib64"), "-Wl,-rpath," + os.path.join(cuda, "lib64"),
              "-lcudart"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
