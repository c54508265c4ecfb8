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
                  os.path.join(CSRC, "pcpd_paper.cuh"),
                  os.path.join(CSRC, "pcpd_jit_src.inc"),
                  os.path.join(os.path.dirname(HERE), "include", "pcpd.h")]


JIT_SRC = os.path.join(CSRC, "pcpd_jit_src.inc")
JIT_PRELUDE = """// runtime-compiled copy of the sweep engine (generated by build.py; do not edit)
#define PCPD_JIT_SOURCE 1
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned long long uint64_t;
typedef long long int64_t;
typedef unsigned long long uintptr_t;
"""
JIT_ENTRY = """
extern "C" __global__ void __launch_bounds__(pcpdk::kSweepThreads, 1) pcpd_jit_sweep(const pcpdk::BatchParams B) {
  pcpdk::sweep_body<false, PCPD_JIT_W>(B);
}
extern "C" __global__ void __launch_bounds__(pcpdk::kSweepThreads, 1) pcpd_jit_sweep_batch(const pcpdk::BatchParams B) {
  pcpdk::sweep_body<true, PCPD_JIT_W>(B);
}
"""


def write_jit_source() -> str:
    """The engine's source as a C string for the runtime compiler (thresholds as constants)."""
    parts = [JIT_PRELUDE]
    for fn in ("pcpd_kernels.cuh", "pcpd_engine.cuh"):
        parts.append(open(os.path.join(CSRC, fn)).read())
    parts.append(JIT_ENTRY)
    body = "\n".join(parts)
    assert ")PCPDJIT\"" not in body
    text = "// generated by build.py from pcpd_kernels.cuh and pcpd_engine.cuh\n" \
           "static const char kJitSource[] = R\"PCPDJIT(" + body + ")PCPDJIT\";\n"
    old = open(JIT_SRC).read() if os.path.exists(JIT_SRC) else None
    if old != text:
        with open(JIT_SRC, "w") as f:
            f.write(text)
    return JIT_SRC


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def flags(extra=()):
    return ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
            "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "--shared", *extra]


DEBUG_LIB = os.path.join(HERE, "libpcpd_debug.so")


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """libpcpd.so; debug=True: libpcpd_debug.so, with every kernel index checked (-DPCPD_DEBUG)."""
    write_jit_source()
    out = DEBUG_LIB if debug else LIB
    stale = force or not os.path.exists(out) or any(
        os.path.getmtime(d) > os.path.getmtime(out) for d in DEPS)
    if stale:
        tmp = out + ".tmp%d" % os.getpid()
        extra = (["-Xptxas", "-v"] if verbose else []) + (["-DPCPD_DEBUG"] if debug else [])
        cmd = [nvcc(), *flags(extra), *SOURCES, "-o", tmp, "-lcudart", "-ldl"]
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


PIPES_LIB = os.path.join(HERE, "libpcpd_pipes.so")
PIPES_SRC = os.path.join(CSRC, "pcpd_pipes.cu")
PIPES_DEPS = [PIPES_SRC, os.path.join(os.path.dirname(HERE), "include", "pcpd_pipes.h")]


def build_pipes(force: bool = False) -> str:
    """libpcpd_pipes.so: the integer-pipe lane-rate kernels behind the roofline peaks."""
    stale = force or not os.path.exists(PIPES_LIB) or any(
        os.path.getmtime(d) > os.path.getmtime(PIPES_LIB) for d in PIPES_DEPS)
    if stale:
        tmp = PIPES_LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc(), *flags(), PIPES_SRC, "-o", tmp, "-lcudart"])
        os.replace(tmp, PIPES_LIB)
    return PIPES_LIB


EXAMPLE_SRC = os.path.join(HERE, "examples", "pcpd_decay.c")
EXAMPLE_BIN = os.path.join(HERE, "examples", "pcpd_decay")


def build_example(force: bool = False) -> str:
    """The plain C example program, linked against the in-tree libpcpd.so (rpath $ORIGIN)."""
    lib = build()
    stale = force or not os.path.exists(EXAMPLE_BIN) or any(
        os.path.getmtime(d) > os.path.getmtime(EXAMPLE_BIN) for d in (EXAMPLE_SRC, lib))
    if stale:
        tmp = EXAMPLE_BIN + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-I", os.path.join(os.path.dirname(HERE), "include"),
                               EXAMPLE_SRC, "-o", tmp, "-L", HERE, "-lpcpd", "-Wl,-rpath,$ORIGIN/..", "-lm"])
        os.replace(tmp, EXAMPLE_BIN)
    return EXAMPLE_BIN


if __name__ == "__main__":
    build(force=True, verbose=True)
    build_pipes(force=True)
