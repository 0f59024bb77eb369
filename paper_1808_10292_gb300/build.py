"""Build the isort shared library (libisort.so) in-tree with nvcc for sm_103a.

Each translation unit under csrc/ is compiled in parallel to an object under
_build/, then linked into paper_1808_10292_gb300/libisort.so (static cudart).
Also builds the seeded input generator (inputs/libsynth.so), which is a
separate library that shares nothing with the sort.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libisort.so")
SYNTH_SRC = os.path.join(ROOT, "inputs", "synth.cu")
SYNTH_LIB = os.path.join(ROOT, "inputs", "libsynth.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found; the isort library needs the CUDA toolkit to build")


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def _sources():
    srcs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    deps = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cuh", ".h"))) + [os.path.join(INCLUDE, "isort.h")]
    return srcs, deps


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build step failed: {' '.join(cmd)}\n{r.stdout}")
    return r.stdout


def build_synth(force: bool = False, verbose: bool = False) -> str:
    if force or not os.path.exists(SYNTH_LIB) or os.path.getmtime(SYNTH_LIB) < os.path.getmtime(SYNTH_SRC):
        tmp = SYNTH_LIB + f".tmp{os.getpid()}"
        _run([nvcc(), *ARCH, *NVCC_FLAGS, "-shared", SYNTH_SRC, "-o", tmp])
        os.replace(tmp, SYNTH_LIB)
        if verbose:
            print("built", SYNTH_LIB)
    return SYNTH_LIB


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a and link libisort.so; returns its path."""
    srcs, deps = _sources()
    os.makedirs(BUILD, exist_ok=True)
    dep_time = _newest(deps)
    jobs = []
    for s in srcs:
        obj = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        if force or ptxas_info or not os.path.exists(obj) or os.path.getmtime(obj) < max(
                os.path.getmtime(s), dep_time):
            cmd = [nvcc(), *ARCH, *NVCC_FLAGS, f"-I{INCLUDE}", "-c", s, "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            outs = list(ex.map(_run, jobs))
        if verbose or ptxas_info:
            for o in outs:
                if o.strip():
                    print(o)
    if jobs or force or not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest(objs):
        tmp = LIB + f".tmp{os.getpid()}"
        _run([nvcc(), *ARCH, "-shared", *objs, "-o", tmp])
        os.replace(tmp, LIB)
        if verbose:
            print("built", LIB)
    build_synth(force=force, verbose=verbose)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
