"""Build libme.so in-tree with nvcc for sm_103a (no cmake, no torch).

Each translation unit under csrc/ compiles in parallel into _build/, then
one link produces paper_1401_5245_gb300/libme.so against the shared CUDA
runtime (the same libcudart.so.13 torch loads).  The serving load
generator (csrc/loadgen/, host code calling libme's C ABI only) becomes
libme_loadgen.so beside it.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libme.so")
LOADGEN_SRC = os.path.join(CSRC, "loadgen", "me_loadgen.cpp")
LOADGEN = os.path.join(PKG, "libme_loadgen.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-Wall", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"),
                 "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) +
                  glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.h")) +
            glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    headers = _headers()
    jobs = []
    objs = []
    for src in _sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or ptxas_info or _stale(obj, [src] + headers):
            extra = ["-Xptxas", "-v"] if ptxas_info else []
            jobs.append([cc] + ARCH + FLAGS + extra + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for cmd, r in ex.map(run, jobs):
                if verbose or r.returncode != 0 or ptxas_info:
                    sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed on {cmd[-3]}")
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [cc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link of libme.so failed")
        os.replace(tmp, LIB)
    build_loadgen(force)
    return LIB


def cxx() -> str:
    for cand in (os.environ.get("CXX"), shutil.which("g++"), shutil.which("c++")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("no C++ compiler found")


def build_loadgen(force: bool = False) -> str:
    """libme_loadgen.so: host code linked against libme.so (found beside it)."""
    deps = [LOADGEN_SRC, os.path.join(INCLUDE, "me.h"), LIB]
    if not (force or _stale(LOADGEN, deps)):
        return LOADGEN
    tmp = LOADGEN + f".tmp{os.getpid()}"
    cmd = [cxx(), "-O3", "-std=c++17", "-shared", "-fPIC", "-Wall", "-I", INCLUDE,
           LOADGEN_SRC, "-o", tmp, "-L", PKG, "-lme", "-Wl,-rpath,$ORIGIN", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        raise RuntimeError("build of libme_loadgen.so failed")
    os.replace(tmp, LOADGEN)
    return LOADGEN


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          ptxas_info="--ptxas-info" in sys.argv)
    print(LIB)
