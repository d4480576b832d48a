"""Build step of the native library: nvcc for sm_103a, in tree.

``build_library()`` compiles ``csrc/vox.cu`` (which includes the kernel headers)
into ``libvox.so`` next to this file. It runs anywhere nvcc runs; no GPU needed.
"""

from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libvox.so")
SOURCES = [os.path.join(CSRC, "vox.cu")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    files = list(SOURCES)
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h")):
                files.append(os.path.join(d, f))
    return files


def needs_build(out: str = LIB) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(f) > t for f in _inputs())


def nvcc_command(out: str = LIB, extra=()):
    nvcc = os.environ.get("NVCC", "nvcc")
    # -cudart shared: the library uses the same CUDA runtime instance (and so the
    # same current device and streams) as the process that loads it, e.g. torch
    return [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
            "-cudart", "shared", "-I", INCLUDE, *extra, "-o", out, *SOURCES]


def build_library(out: str = LIB, force: bool = False, verbose: bool = False, extra=()) -> str:
    if force or needs_build(out):
        cmd = nvcc_command(out, extra)
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
    return out
