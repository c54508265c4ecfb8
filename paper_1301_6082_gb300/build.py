"""Builds libpcpd.so in-tree with nvcc for sm_103a (no CPU fallback is built)."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpcpd.so")
SOURCES = [os.path.join(CSRC, "pcpd_capi.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "pcpd_kernels.cuh"), os.path.join(CSRC, "pcpd_engine.cuh"),
                  os.path.join(os.path.dirname(HERE), "include", "pcpd.h")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def flags(extra=()):
    return ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
            "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "--shared", *extra]


def build(force: bool = False, verbose: bool = False) -> str:
    stale = force or not os.path.exists(LIB) or any(
        os.path.getmtime(d) > os.path.getmtime(LIB) for d in DEPS)
    if stale:
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc(), *flags(["-Xptxas", "-v"] if verbose else []), *SOURCES, "-o", tmp, "-lcudart"]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
