"""Build libfsi.so (the CUDA library) in-tree for sm_103a with nvcc.

    python -m paper_2210_02472_b300.build [--verbose-ptxas]
"""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
LIB = PKG / "libfsi.so"
INCLUDE = PKG.parent / "include"
SOURCES = ["pair_kernels.cu", "aux_kernels.cu", "vjp_kernels.cu", "batch_kernels.cu", "hhs_small.cu", "hhs_grid.cu", "order_kernels.cu", "noalloc.cu", "probe_kernels.cu", "subsys_kernels.cu", "steps_x2.cu", "steps_f64.cu", "fsi_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    return cand if Path(cand).exists() else "nvcc"


def build(force: bool = False, verbose_ptxas: bool = False) -> Path:
    srcs = [CSRC / s for s in SOURCES]
    deps = srcs + [CSRC / "fsi_internal.cuh", CSRC / "pair_math.cuh", CSRC / "sym_x2.cuh", CSRC / "hhs_small.cuh", INCLUDE / "fsi.h"]
    if not force and LIB.exists() and all(LIB.stat().st_mtime >= d.stat().st_mtime for d in deps):
        return LIB
    objdir = PKG / "_build"
    objdir.mkdir(exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I", str(INCLUDE), "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        flags += ["-Xptxas", "-v"]
    objs = []
    for s in srcs:
        o = objdir / (s.stem + ".o")
        subprocess.check_call([nvcc()] + flags + ["-c", str(s), "-o", str(o)])
        objs.append(str(o))
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
    subprocess.check_call([nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", str(tmp)] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose_ptxas="--verbose-ptxas" in sys.argv)
    print(LIB)
