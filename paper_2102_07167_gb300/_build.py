"""Builds libkura.so in-tree: the CUDA translation unit for sm_103a (nvcc) and
the host planner (g++ with OpenMP), compiled in parallel, linked with nvcc."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libkura.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkura.so")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cpp", ".cuh", ".hpp"))] + [os.path.join(INCLUDE, "kura.h")]


def build_library(force: bool = False, verbose: bool = False) -> str:
    srcs = _sources()
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in srcs):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", INCLUDE, "-I", CSRC]
    cu_srcs = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    objs, cmds = [], []
    for f in cu_srcs:
        o = os.path.join(BUILD, f[:-3] + ".o")
        objs.append(o)
        cmds.append([nvcc, ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp", *inc,
                     "-Xptxas", "-v" if verbose else "-O3", "-c", os.path.join(CSRC, f), "-o", o])
    cpp_obj = os.path.join(BUILD, "plan.o")
    objs.append(cpp_obj)
    cmds.append(["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", *inc, "-c", os.path.join(CSRC, "plan.cpp"),
                 "-o", cpp_obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"build step failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stdout + r.stderr

    with ThreadPoolExecutor(len(cmds)) as ex:
        outs = list(ex.map(run, cmds))
    if verbose:
        print("".join(outs))
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc, ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"])
    os.replace(tmp, LIB)
    return LIB


def kernel_source_hash() -> str:
    """Hash of the source of the row and trig kernels (kura_kernels.cuh): profile records made from other
    sources are stale."""
    import hashlib
    h = hashlib.sha256()
    with open(os.path.join(CSRC, "kura_kernels.cuh"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]
