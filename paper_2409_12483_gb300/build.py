"""Build the sm_103a shared library libader_gb300.so in-tree.

One nvcc translation unit per degree N (ader_deg.cu with -DADER_DEG=N), the C
ABI (ader_capi.cu) and the host operator construction (ader_ops.cpp), compiled
in parallel and linked with nvcc.  No CPU fallback is built: the library is the
only compute path.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libader_gb300.so")
DEGREES = range(0, 8)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]


def _nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libader_gb300.so")
    return path


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [
        os.path.join(INCLUDE, "ader.h")]


def _jobs():
    nvcc = _nvcc()
    jobs = []
    for d in DEGREES:
        obj = os.path.join(BUILD, f"ader_deg{d}.o")
        jobs.append((obj, [nvcc, *ARCH, *NVCC_FLAGS, f"-DADER_DEG={d}", "-c",
                           os.path.join(CSRC, "ader_deg.cu"), "-o", obj]))
    for name in ("ader_capi", "ader_server"):
        obj = os.path.join(BUILD, f"{name}.o")
        jobs.append((obj, [nvcc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, f"{name}.cu"), "-o", obj]))
    obj = os.path.join(BUILD, "ader_ops.o")
    jobs.append((obj, [nvcc, *NVCC_FLAGS, "-x", "c++", "-c", os.path.join(CSRC, "ader_ops.cpp"),
                       "-o", obj]))
    return jobs


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    jobs = _jobs()

    def run(job):
        obj, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    workers = max(1, min(len(jobs), os.cpu_count() or 4))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(run, jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
