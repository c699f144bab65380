"""In-tree build of libisg.so (CUDA, sm_103a) with nvcc; no CMake, no torch headers.

Translation units compile in parallel; a unit is rebuilt when it or any
header under ``csrc/`` or ``include/`` is newer than its object file.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libisg.so")

SOURCES = ["isg_runtime.cu", "isg_batch.cu", "isg_server.cu", "torus_msc.cu", "csr_sweep.cu",
           "aux_kernels.cu", "isg_noalloc.cu", "csr_msc.cu", "csr_msc_fields.cu",
           "pipe_peaks.cu", "tempering.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libisg")


def _cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def _headers():
    hs = []
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".h", ".cuh")):
                hs.append(os.path.join(d, f))
    return hs


def _flags(extra_ptxas: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if extra_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every CUDA translation unit and link libisg.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(os.path.join(BUILD, "obj"), exist_ok=True)
    newest_header = max(os.path.getmtime(h) for h in _headers())
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, "obj", src.replace(".cu", ".o"))
        objs.append(o)
        if force or ptxas_info or not os.path.exists(o) or \
                os.path.getmtime(o) < max(os.path.getmtime(s), newest_header):
            jobs.append((s, o))

    def compile_one(job):
        s, o = job
        tmp = o + f".tmp{os.getpid()}"
        cmd = [nvcc, "-c", s, "-o", tmp] + _flags(ptxas_info)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(s)}:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, o)
        return s, res.stderr

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for s, err in ex.map(compile_one, jobs):
                if verbose or ptxas_info:
                    sys.stderr.write(f"[{os.path.basename(s)}]\n{err}")
    if jobs or force or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + [
            "-cudart", "shared", "-Xlinker", "-rpath," + _cuda_lib_dir(nvcc)]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"linking libisg.so failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
