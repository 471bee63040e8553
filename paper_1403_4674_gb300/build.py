"""Build the sm_103a shared library in-tree (no torch extension machinery).

    python -m paper_1403_4674_gb300.build

Produces paper_1403_4674_gb300/_build/libkmc_gb300.so from csrc/*.cu with
nvcc -gencode arch=compute_103a,code=sm_103a; host code is compiled without
floating-point contraction so that the host rate table is bit-stable across
x86-64 and aarch64.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libkmc_gb300.so")
SOURCES = [os.path.join(CSRC, "kmc_api.cu")]
DEPS = SOURCES + [os.path.join(CSRC, name) for name in ("kmc_kernels.cuh", "kmc_ring.cuh", "kmc_part.cuh",
                                                          "kmc_tpd.cuh", "kmc_tpdr.cuh", "kmc_tpdr64.cuh")] + \
    [os.path.join(ROOT, "include", "kmc.h")]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return cand


def command(out: str, verbose_ptxas: bool = False) -> list[str]:
    cmd = [nvcc(), "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
           "-shared", "-cudart", "shared", "-Xcompiler", "-fPIC,-ffp-contract=off",
           "-I", os.path.join(ROOT, "include"), "-o", out] + SOURCES
    if verbose_ptxas:
        cmd.insert(1, "-Xptxas=-v")
    return cmd


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in DEPS)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and not verbose_ptxas and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = command(tmp, verbose_ptxas)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed building %s" % LIB)
    if verbose_ptxas:
        sys.stderr.write(res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose_ptxas="-v" in sys.argv)
    print(LIB)
