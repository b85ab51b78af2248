"""Builds the CUDA library ``libpac.so`` for sm_103a (GB300) in-tree.

Each ``csrc/*.cu`` file is compiled by nvcc in parallel, then linked into one
shared library with the CUDA runtime linked statically, so the library loads
on any machine with the driver (and, without a GPU, still loads for symbol
checks).  No CMake.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libpac.so")
# synthetic-input generator for benchmarks and tests: a library of its own,
# so the method's library holds nothing but the method
GEN_SRC = os.path.join(CSRC, "gen")
GEN_LIB = os.path.join(HERE, "libpacgen.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              f"-I{INCLUDE}", f"-I{CSRC}"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compiles and links libpac.so and libpacgen.so if any source changed;
    returns the path of libpac.so."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    headers = _headers()
    srcs = _sources()
    gen_srcs = sorted(glob.glob(os.path.join(GEN_SRC, "*.cu")))
    objs, gen_objs = [], []
    jobs = []
    for src in srcs + gen_srcs:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        (gen_objs if src in gen_srcs else objs).append(obj)
        if force or _stale(obj, [src] + headers):
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", obj]
            jobs.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return r

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    for lib, lib_objs in ((LIB, objs), (GEN_LIB, gen_objs)):
        if lib_objs and (force or jobs or _stale(lib, lib_objs)):
            tmp = lib + f".tmp{os.getpid()}"
            run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *lib_objs])
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
