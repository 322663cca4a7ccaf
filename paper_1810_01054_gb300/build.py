"""Builds libgbmpm.so in-tree (paper_1810_01054_gb300/_build/) with nvcc for sm_103a.

Usage: ``python -m paper_1810_01054_gb300.build [--force]``.  Translation units compile in
parallel; the link is skipped when nothing changed.
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgbmpm.so")
SOURCES = ["mpm_kernels.cu", "mpm_ctrl.cu", "mpm_api.cu", "mpm_batch.cu", "mpm_noalloc.cu", "mpm_tune.cu", "mpm_f64.cu"]
HEADERS = ["mpm_device.cuh", "mpm_internal.h", "mpm_scene.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgbmpm")


def _mtime(p: str) -> float:
    return os.path.getmtime(p) if os.path.exists(p) else -1.0


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "mpm.h")]
    dep_t = max(_mtime(d) for d in deps)
    jobs = []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or _mtime(obj) < max(_mtime(sp), dep_t):
            jobs.append((sp, obj))

    def compile_one(job):
        sp, obj = job
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, *FLAGS, "-c", sp, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(sp)}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, obj)
        if verbose:
            print("compiled", os.path.basename(sp), file=sys.stderr)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(compile_one, jobs))
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    if jobs or force or _mtime(LIB) < max(_mtime(o) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
