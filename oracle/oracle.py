"""Python face of the plain CPU oracle (``pcpd_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The product library never imports this module.

The oracle follows the paper (Schram, arXiv 1301.6082): Eq. (1) rates, Alg. 1's decision
tree applied on random-phase 3-site windows, integer thresholds floor(rate*2^32) (the
exact form of the dyadic masks of Sec. 4.2-4.3), Philox4x32-10 random bits.  The
per-function citations are in the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcpd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_FULL, MODE_EMPTY, MODE_HALF = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, plain -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            u8p, u32p, u64p = C.POINTER(C.c_uint8), C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_philox_batch.argtypes = [u32p, C.c_uint64, u32p, C.c_uint64]
            L.orc_thresholds.argtypes = [C.c_double, C.c_double, u64p, u64p, u64p]
            L.orc_thresholds.restype = C.c_int
            L.orc_substep_of_time.argtypes = [C.c_uint32, C.c_uint64]
            L.orc_substep_of_time.restype = C.c_uint64
            L.orc_substep_of_time_w.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64]
            L.orc_substep_of_time_w.restype = C.c_uint64
            L.orc_phase.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
            L.orc_phase.restype = C.c_uint32
            L.orc_init.argtypes = [u8p, C.c_uint32, C.c_uint32, C.c_int, C.c_uint64, C.c_uint32]
            L.orc_init.restype = C.c_int
            L.orc_run.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint64, u8p,
                                  C.c_uint64, C.c_uint64, u64p, C.c_uint32, u64p, u32p, u64p, C.c_int, C.c_uint32, u64p,
                                  C.c_uint32]
            L.orc_run.restype = C.c_int
            L.orc_rs_run.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint64, u8p,
                                     C.c_uint64, C.c_uint64, u64p, C.c_uint32, u64p, u32p, C.c_int]
            L.orc_rs_run.restype = C.c_int
            L.orc_paper_run.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                        C.c_uint32, C.c_uint64, C.c_uint64, u8p, C.c_uint64, C.c_uint64,
                                        u64p, C.c_uint32, u64p, C.c_uint32, u32p]
            L.orc_paper_run.restype = C.c_int
            L.orc_pack.argtypes = [u8p, C.c_uint32, C.c_uint32, u32p]
            L.orc_unpack.argtypes = [u32p, C.c_uint32, C.c_uint32, u8p]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def philox(ctrs, seed: int) -> np.ndarray:
    """Philox4x32-10 blocks for counters ``ctrs`` ([n,4] uint32) under key = seed."""
    c = np.ascontiguousarray(ctrs, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(c)
    lib().orc_philox_batch(_p(c, C.c_uint32), C.c_uint64(seed), _p(out, C.c_uint32), c.shape[0])
    return out


def thresholds(p: float, d: float):
    """(T_D, T_DA, T_P) as Python ints (R3, R11)."""
    td, tda, tp = C.c_uint64(), C.c_uint64(), C.c_uint64()
    if lib().orc_thresholds(p, d, C.byref(td), C.byref(tda), C.byref(tp)) != 0:
        raise ValueError("p, d must lie in [0, 1]")
    return int(td.value), int(tda.value), int(tp.value)


def substep_of_time(L: int, t: int, tuple_n: int = 2) -> int:
    """Sub-step at which MCS time t is reached: ceil(t*L/K), K = floor(L/(n+1))."""
    if tuple_n == 2:
        return int(lib().orc_substep_of_time(L, t))
    return int(lib().orc_substep_of_time_w(L, tuple_n + 1, t))


def phase(seed: int, L: int, h: int, n: int) -> int:
    return int(lib().orc_phase(seed, L, h, n))


def init_state(L: int, S: int, mode: int = MODE_FULL, seed: int = 1, group0: int = 0) -> np.ndarray:
    """Initial byte state [S][L] of groups group0 .. group0 + S/32 - 1 of an instance."""
    st = np.zeros((S, L), dtype=np.uint8)
    if lib().orc_init(_p(st, C.c_uint8), L, S, mode, seed, group0) != 0:
        raise ValueError("bad init arguments")
    return st


def pack(state: np.ndarray) -> np.ndarray:
    """Byte state [S][L] -> canonical words u32 [S/32][L]."""
    st = np.ascontiguousarray(state, dtype=np.uint8)
    S, L = st.shape
    w = np.zeros((S // 32, L), dtype=np.uint32)
    lib().orc_pack(_p(st, C.c_uint8), L, S, _p(w, C.c_uint32))
    return w


def unpack(words: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32)
    G, L = w.shape
    st = np.zeros((32 * G, L), dtype=np.uint8)
    lib().orc_unpack(_p(w, C.c_uint32), L, 32 * G, _p(st, C.c_uint8))
    return st


def run(state: np.ndarray, p: float, d: float, seed: int, n_begin: int, n_end: int,
        rec_sub=(), per_sample: bool = False, threads: int | None = None, group0: int = 0,
        pairs: bool = False, tuple_n: int = 2):
    """Advance ``state`` (modified in place, [S][L] bytes: groups group0, group0+1, ... of an
    instance) from sub-step n_begin to n_end on the window schedule; tuple_n = 2 (PCPD),
    3 (TCPD) or 4 (QCPD), windows of tuple_n + 1 sites.
    Returns (totals u64[R], per-sample u32[R][S] or None, events[3]), plus the occupied
    nearest-neighbour pair counts u64[R] as a fourth element when ``pairs``."""
    assert state.dtype == np.uint8 and state.flags.c_contiguous
    S, L = state.shape
    td, tda, _ = thresholds(p, d)
    rec = np.ascontiguousarray(rec_sub, dtype=np.uint64)
    tot = np.zeros(len(rec), dtype=np.uint64)
    ps = np.zeros((len(rec), S), dtype=np.uint32) if per_sample else None
    ev = np.zeros(3, dtype=np.uint64)
    prs = np.zeros(len(rec), dtype=np.uint64)
    nt = threads if threads is not None else (os.cpu_count() or 1)
    rc = lib().orc_run(L, S, td, tda, C.c_uint64(seed), _p(state, C.c_uint8), n_begin, n_end,
                       _p(rec, C.c_uint64), len(rec), _p(tot, C.c_uint64),
                       _p(ps, C.c_uint32) if ps is not None else None, _p(ev, C.c_uint64), nt, group0,
                       _p(prs, C.c_uint64), tuple_n)
    if rc == 2:
        raise AssertionError("oracle: a window changed the particle number by other than +1, -n, 0")
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    if pairs:
        return tot, ps, ev, prs
    return tot, ps, ev


def rs_run(state: np.ndarray, p: float, d: float, seed: int, a_begin: int, a_end: int,
           rec_att=(), per_sample: bool = False, threads: int | None = None):
    """Alg. 1 random-sequential attempts [a_begin, a_end) on ``state`` (in place)."""
    assert state.dtype == np.uint8 and state.flags.c_contiguous
    S, L = state.shape
    td, _, tp = thresholds(p, d)
    rec = np.ascontiguousarray(rec_att, dtype=np.uint64)
    tot = np.zeros(len(rec), dtype=np.uint64)
    ps = np.zeros((len(rec), S), dtype=np.uint32) if per_sample else None
    nt = threads if threads is not None else (os.cpu_count() or 1)
    rc = lib().orc_rs_run(L, S, td, tp, C.c_uint64(seed), _p(state, C.c_uint8), a_begin, a_end,
                          _p(rec, C.c_uint64), len(rec), _p(tot, C.c_uint64),
                          _p(ps, C.c_uint32) if ps is not None else None, nt)
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    return tot, ps


def paper_thresholds(p: float, d: float, m: int, n_dec: int):
    """(T_d, T_c) of the paper's scheme: d must be a multiple of 2^-m (T_d = d*2^m), and
    p*2^n_dec <= 1 (T_c = floor(p*2^n_dec*2^32), 2^32 meaning always); m, n_dec <= 16."""
    if not (0 <= m <= 16 and 0 <= n_dec <= 16):
        raise ValueError("m and n_dec must lie in [0, 16]")
    td = d * (1 << m)
    if td != int(td) or not (0 <= td <= (1 << m)):
        raise ValueError("d must be a multiple of 2^-m in [0, 1]")
    c = p * float(1 << n_dec)
    if not (0.0 <= c <= 1.0):
        raise ValueError("need 0 <= p * 2^n_dec <= 1")
    tc = min(1 << 32, int(np.floor(c * 4294967296.0)))
    return int(td), tc


def paper_run(state: np.ndarray, n_loc: int, S_w: int, p: float, d: float, m: int, n_dec: int,
              seed: int, step_begin: int, step_end: int, rec_step=(), sys0: int = 0,
              per_system: bool = False):
    """The paper's shared-local-site scheme (Sec. 3-4, Alg. 2) on ``state`` [systems][L]
    bytes (systems sys0, sys0+1, ...), L = 32*n_loc*S_w, in place.  Returns the record
    totals, and the per-system counts [n_rec][systems] when ``per_system``."""
    st = state
    assert st.dtype == np.uint8 and st.flags.c_contiguous and st.shape[1] == 32 * n_loc * S_w
    td, tc = paper_thresholds(p, d, m, n_dec)
    rec = np.ascontiguousarray(rec_step, dtype=np.uint64)
    tot = np.zeros(len(rec), dtype=np.uint64)
    ps = np.zeros((len(rec), st.shape[0]), dtype=np.uint32)
    rc = lib().orc_paper_run(n_loc, S_w, st.shape[0], m, td, n_dec, tc, C.c_uint64(seed), _p(st, C.c_uint8),
                             step_begin, step_end, _p(rec, C.c_uint64), len(rec), _p(tot, C.c_uint64),
                             sys0, _p(ps, C.c_uint32))
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    return (tot, ps) if per_system else tot
