"""Build the in-tree CUDA library ``_lib/librsa_gb300.so`` for sm_103a.

The library has two translation units, compiled in parallel and linked
together: ``csrc/rsa.cu`` (the engine: handles, round, contact-graph and
first-wrap kernels) and ``csrc/rsa_mix.cu`` (samples of uneven shapes: the
small-lattice one-CTA-per-sample kernel, mixed batches, the autotuner)."""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
SRC = os.path.join(CSRC, "rsa.cu")
SOURCES = [SRC, os.path.join(CSRC, "rsa_mix.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in (
    "rsa_kernels.cuh", "rsa_device.cuh", "rsa_tile.cuh", "rsa_line.cuh", "rsa_lwin.cuh",
    "rsa_config.cuh", "rsa_small.cuh")] + [os.path.join(os.path.dirname(HERE), "include", "rsa.h")]
LIB = os.path.join(HERE, "_lib", "librsa_gb300.so")
OBJ_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMPILE_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                        "-Xcompiler", "-O2"]
NVCC_FLAGS = COMPILE_FLAGS + ["-shared"]  # one-step form (single source)


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    os.makedirs(OBJ_DIR, exist_ok=True)
    stale = not os.path.exists(LIB) or any(
        os.path.getmtime(d) > os.path.getmtime(LIB) for d in DEPS)
    if not (force or stale):
        return LIB
    pid = os.getpid()
    objs = [os.path.join(OBJ_DIR, os.path.basename(s) + ".%d.o" % pid) for s in SOURCES]

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [nvcc()] + COMPILE_FLAGS + (["-Xptxas", "-v"] if verbose else []) + \
            ["-c", "-o", obj, src]
        subprocess.check_call(cmd)

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        list(ex.map(compile_one, zip(SOURCES, objs)))
    tmp = LIB + ".tmp.%d" % pid
    subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
