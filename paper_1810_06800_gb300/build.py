"""Build the in-tree CUDA library ``_lib/librsa_gb300.so`` for sm_103a."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "rsa.cu")
DEPS = [SRC, os.path.join(HERE, "csrc", "rsa_kernels.cuh"),
        os.path.join(HERE, "csrc", "rsa_device.cuh"), os.path.join(HERE, "csrc", "rsa_tile.cuh"),
        os.path.join(HERE, "csrc", "rsa_line.cuh"), os.path.join(HERE, "csrc", "rsa_lwin.cuh"),
        os.path.join(HERE, "csrc", "rsa_config.cuh"),
        os.path.join(os.path.dirname(HERE), "include", "rsa.h")]
LIB = os.path.join(HERE, "_lib", "librsa_gb300.so")
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
              "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    stale = not os.path.exists(LIB) or any(
        os.path.getmtime(d) > os.path.getmtime(LIB) for d in DEPS)
    if force or stale:
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = [nvcc()] + NVCC_FLAGS + (["-Xptxas", "-v"] if verbose else []) + ["-o", tmp, SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
