"""Builds the planner's CUDA library (libplan.so) in-tree for sm_103a.

The library is plain CUDA C++ behind the C ABI of include/plan.h; no torch
headers are involved, so one nvcc call builds it in a few seconds.

    python -m paper_1311_4527_gb300.build
"""
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libplan.so")
SOURCES = [os.path.join(CSRC, "plan.cu")]
DEPS = SOURCES + [os.path.join(CSRC, n) for n in ("twa_math.cuh", "twa_iter.cuh", "twa_adjoint.cuh",
                                                  "twa_backward.cuh")] + [os.path.join(INCLUDE, "plan.h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc_path():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the planner's CUDA library cannot be built")


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile libplan.so unless it is newer than every source.  Returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    tmp = LIB + ".tmp"
    cmd = [nvcc_path(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-shared", "-I", INCLUDE, "-I", CSRC, "-o", tmp, *SOURCES, *extra_flags]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else []))
