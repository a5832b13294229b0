"""Build libboltz.so in-tree for sm_103a (GB300).

Two translation units compiled in parallel (the CUDA one with nvcc, the host
quadrature with g++), then linked into paper_2112_02695_gb300/libboltz.so.
Usage:  python -m paper_2112_02695_gb300.build  [--force]
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libboltz.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cpp", ".cuh", ".hpp"))] + [os.path.join(ROOT, "include", "boltz.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    obj_cu = os.path.join(BUILD, "boltz.o")
    obj_cpp = os.path.join(BUILD, "quadrature.o")
    cmds = [
        [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
         *inc, "-c", os.path.join(CSRC, "boltz.cu"), "-o", obj_cu],
        ["g++", "-O2", "-std=c++17", "-fPIC", *inc, "-c", os.path.join(CSRC, "quadrature.cpp"), "-o", obj_cpp],
    ]

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=2) as ex:
        results = list(ex.map(run, cmds))
    for cmd, r in results:
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            sys.stderr.write(r.stderr)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as fh:
        fh.write(results[0][1].stderr)
    link = [_nvcc(), *ARCH, "-shared", "-o", LIB + ".tmp", obj_cu, obj_cpp, "-lcudart"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + " ".join(link) + "\n" + r.stdout + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
