"""Build libegt.so in-tree with nvcc for sm_103a (B300), and libegt_cpu.so (the
FP64 multi-core CPU comparator) with g++ and OpenMP.

Usage: ``python -m paper_1810_03063_b300.build [--force]``.  Objects go to
``_build/`` at the repository root; the shared libraries are written next to
this file so that they travel with the source tree.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libegt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "-Xcompiler", "-fvisibility=hidden",
         "-I", INCLUDE]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".hpp", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


CPU_LIB = os.path.join(PKG, "libegt_cpu.so")
CPU_SRC = [os.path.join(PKG, "cpu", "egt_cpu.cpp"), os.path.join(CSRC, "tree.cpp")]
CPU_HDR = [os.path.join(INCLUDE, "egt.h"), os.path.join(INCLUDE, "egt_cpu.h"), os.path.join(CSRC, "tree.hpp")]


def build_cpu(force: bool = False) -> str:
    """The FP64 multi-core CPU comparator (include/egt_cpu.h): g++ with OpenMP, x86-64-v3."""
    newest = max(os.path.getmtime(f) for f in CPU_SRC + CPU_HDR)
    if not force and os.path.exists(CPU_LIB) and os.path.getmtime(CPU_LIB) >= newest:
        return CPU_LIB
    cxx = os.environ.get("CXX") or shutil.which("g++") or "g++"
    cmd = [cxx, "-O3", "-march=x86-64-v3", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-fvisibility=hidden",
           "-I", INCLUDE, *CPU_SRC, "-o", CPU_LIB]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"g++ failed on the CPU comparator:\n{res.stdout}\n{res.stderr}")
    return CPU_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    hdr_time = max(os.path.getmtime(h) for h in headers())
    objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        if (not force and os.path.exists(obj) and os.path.getmtime(obj) >= os.path.getmtime(src)
                and os.path.getmtime(obj) >= hdr_time):
            continue
        cmd = [nvcc, *ARCH, *FLAGS, "-Xptxas", "-v", "-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, *FLAGS, "-x", "cu", *ARCH, "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        if verbose:
            sys.stderr.write(res.stderr)
    build_cpu(force)
    if force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", LIB, *objs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    return LIB


if __name__ == "__main__":
    path = build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(path)
