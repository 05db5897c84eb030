"""Compile the CUDA/C++ sources into the in-tree shared library ``libspand.so``.

One ``-gencode`` (sm_103a), translation units compiled in parallel, no cmake.
Run as ``python -m paper_2007_00789_gb300.build`` or through
``__graft_entry__.build()``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libspand.so")

# (source, extra flags): the factor/apply translation units are compiled once per precision
_F32 = ["-DSPAND_REAL=float", "-DSPAND_NS=f32", "-DSPAND_SINGLE=1"]
_F64 = ["-DSPAND_REAL=double", "-DSPAND_NS=f64"]
SOURCES = [
    ("symbolic.cpp", []), ("host_pool.cpp", []), ("api.cu", []), ("spand_pcg.cu", []), ("engine.cu", []), ("probe.cu", []),
    ("factor_core.cu", _F64), ("factor_core.cu", _F32),
    ("spand_kernels.cu", _F64), ("spand_kernels.cu", _F32),
    ("spand_apply.cu", _F64), ("spand_apply.cu", _F32),
]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libspand.so")
    return path


def _compile(item, extra: list[str]) -> str:
    src, flags = item
    tag = "_f32" if "-DSPAND_NS=f32" in flags else ("_f64" if flags else "")
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + tag + ".o")
    cmd = [nvcc(), *ARCH, *COMMON, *flags, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc(), *COMMON, *flags, *extra, "-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    return obj


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    """Build libspand.so in place and return its path."""
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra or [])
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"linking failed:\n{' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
