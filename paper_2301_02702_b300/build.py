"""Build libkoma.so in-tree with nvcc for sm_103a.

``python -m paper_2301_02702_b300.build`` (or ``build()``) compiles the CUDA
kernels and the host runtime into ``paper_2301_02702_b300/libkoma.so``. The
library links the shared CUDA runtime (libcudart.so.13), so inside a process
that already loaded PyTorch it uses the same runtime instance.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libkoma.so")
SOURCES = [os.path.join(CSRC, "koma_kernels.cu"), os.path.join(CSRC, "koma_runtime.cpp"),
           os.path.join(CSRC, "koma_server.cpp")]
HEADERS = [os.path.join(CSRC, "koma_internal.h"), os.path.join(CSRC, "koma_host.h"), os.path.join(INCLUDE, "koma.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkoma")
    return cand


def command(out: str = LIB, extra=()):
    return [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-shared",
            "-cudart", "shared", "-I", INCLUDE, "-I", CSRC, *extra, "-o", out, *SOURCES,
            "-Xlinker", "-rpath,/usr/local/cuda/lib64"]


def up_to_date(out: str = LIB) -> bool:
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(p) <= t for p in SOURCES + HEADERS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = command(tmp, ("-Xptxas", "-v") if verbose else ())
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
