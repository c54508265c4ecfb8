"""Measured lane rates of the SM's integer pipes (ctypes binding of libpcpd_pipes.so,
declared in include/pcpd_pipes.h): the denominators of the sweep's roofline.

Each rate is lane-operations completed per SM per clock cycle on the current device, from
one CTA per SM running independent dependency chains of one operation (clock64 around the
timed loop).  Philox rates are in Philox4x32-10 blocks per SM per clock.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpcpd_pipes.so")

OPS = ["lop3", "lop3_2r", "imad_lo", "imad_lo_1r", "imad_hi", "imad_wide", "iadd3", "mix_imad_lo_lop3",
       "mix_light", "mix_imad_wide_lop3", "philox"]
# loop iterations per op: each launch runs a few milliseconds
_ITERS = {"philox": 2000}

_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built (run build.build_pipes())")
        lib = C.CDLL(LIB_PATH)
        lib.pcpd_pipe_rate.argtypes = [C.c_int, C.c_uint32, C.c_uint32, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]
        lib.pcpd_pipe_rate.restype = C.c_int
        lib.pcpd_pipe_count.restype = C.c_int
        assert lib.pcpd_pipe_count() == len(OPS)
        _lib = lib
    return _lib


def rate(op: str, iters: int | None = None, threads: int = 1024) -> tuple[float, float]:
    """(lane-operations per SM per clock, launch milliseconds) of one operation."""
    r, ms = C.c_double(), C.c_double()
    rc = load().pcpd_pipe_rate(OPS.index(op), iters or _ITERS.get(op, 1000), threads, C.byref(r), C.byref(ms))
    if rc != 0:
        raise RuntimeError(f"pcpd_pipe_rate({op}) failed with code {rc}")
    return r.value, ms.value


def all_rates(threads: int = 1024) -> dict:
    """Every operation's rate; Philox blocks are also converted to wide products (20 per
    block) for comparison with the widening-multiply rate."""
    out = {}
    for op in OPS:
        v, ms = rate(op, threads=threads)
        out[op] = round(v, 2)
    out["philox_products"] = round(20.0 * out["philox"], 2)
    return out


if __name__ == "__main__":
    import json
    import sys
    import torch
    torch.cuda.init()
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else 1024
    print(json.dumps({"threads": threads, "lanes_per_sm_clock": all_rates(threads)}))
