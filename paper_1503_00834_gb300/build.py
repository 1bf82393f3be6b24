"""Build libchorus.so in-tree with nvcc for sm_103a (GB300).

Usage: python -m paper_1503_00834_gb300.build   (or build() from Python)
Compiles each translation unit in parallel into _build/ and links the shared library next to
this file.  Objects are rebuilt when their source or a header is newer.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libchorus.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]
SOURCES = ["capi.cu", "batch.cu", "batch_persist.cu", "closure.cu", "closure_tc.cu", "kern_p2.cu", "kern_p3.cu", "kern_p4.cu", "kern_p5.cu", "mesh_builder.cpp"]
# Per-source options.  p = 3: the FP32 square roots (face normals, sound speeds, gravity) use the
# approximate square root (the FP32 perturbation form's tolerance is 1e-5 relative; the FP64 kernels
# are unaffected): 8 % faster there, slower at the other orders, which keep the IEEE square root.
EXTRA_FLAGS = {"kern_p3.cu": ["-prec-sqrt=false"]}


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libchorus")


def _headers_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    paths.append(os.path.abspath(__file__))
    paths.append(os.path.join(INCLUDE, "chorus.h"))
    return max(os.path.getmtime(p) for p in paths)


def _compile(nvcc: str, src: str, hdr_time: float, verbose: bool) -> str:
    obj = os.path.join(BUILD, src + ".o")
    path = os.path.join(CSRC, src)
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(path), hdr_time):
        return obj
    if src.endswith(".cpp"):
        cmd = [nvcc, "-x", "c++", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp", "-I", CSRC, "-I", INCLUDE,
               "-c", path, "-o", obj]
    else:
        cmd = [nvcc] + ARCH + NVFLAGS + EXTRA_FLAGS.get(src, []) + ["-c", path, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return obj


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    hdr = _headers_mtime()
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, hdr, verbose), SOURCES))
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lgomp"]
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
