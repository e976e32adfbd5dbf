"""Builds libdpso_gb300.so in-tree from csrc/ with nvcc for sm_103a.

Each translation unit compiles in parallel; the cost-matrix unit also gets
-fmad=false so no FP64 multiply-add is ever contracted.  The CUDA runtime is
linked statically, so loading the library needs no GPU.
"""
from __future__ import annotations

import concurrent.futures
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
MACHINE = platform.machine()
BUILD = os.path.join(ROOT, "_build", MACHINE)
LIB = os.path.join(HERE, "libdpso_gb300.so")
STAMP = LIB + ".machine"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                 "-I", os.path.join(ROOT, "include")]
SOURCES = {
    "cost.cu": ["-fmad=false"],
    "swarm.cu": [],
    "two_opt.cu": [],
    "two_opt_tiled.cu": [],
    "node_swap_tiled.cu": [],
    "runtime.cu": [],
    "two_opt_noalloc.cu": [],
    "probe.cu": [],
    "server.cu": [],
    "astar.cu": ["-fmad=false"],
}


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return exe


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _lib_matches_machine() -> bool:
    try:
        with open(STAMP) as fh:
            return fh.read().strip() == MACHINE
    except OSError:
        return False


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not _lib_matches_machine():
        force = True
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers.append(os.path.join(ROOT, "include", "dpso.h"))
    jobs = []
    objs = []
    for src, extra in SOURCES.items():
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [path] + headers):
            jobs.append([nvcc(), *COMMON, *extra, "-c", path, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
        with open(STAMP, "w") as fh:
            fh.write(MACHINE + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
