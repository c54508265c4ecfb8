"""Seeded synthetic workloads shaped like the paper's runs (Sec. 5: fully occupied decay
runs, log-spaced density records; lattice sizes, rates and run counts of Sec. 5.3).

This module holds inputs only -- lattice sizes, sample counts, rates, seeds, record times,
instance and request mixes.  It holds none of the method's arithmetic; both the CUDA path
and the CPU oracle take their inputs from here.
"""
from __future__ import annotations

import math

import numpy as np

INIT_FULL, INIT_EMPTY, INIT_HALF = 0, 1, 2


def log_times(t_max: int, n: int) -> list[int]:
    """n strictly increasing integer MCS times, t_k = ceil(t_max^(k/(n-1))), bumped to
    t_{k-1}+1 where rounding would repeat a time."""
    out: list[int] = []
    for k in range(n):
        t = math.ceil(t_max ** (k / (n - 1))) if n > 1 else t_max
        if out and t <= out[-1]:
            t = out[-1] + 1
        out.append(int(t))
    return out


# The single-instance workloads (name -> parameters).
SMALL_L1024 = dict(name="pcpd_L1024_S64", L=1024, S=64, runs=[(0.5, 0.15)], mcs=2000,
                   n_rec=32, seed=1, init=INIT_FULL)
SMEM_L65536 = dict(name="pcpd_L65536_S4096_x3", L=65536, S=4096,
                   runs=[(0.1, 0.11), (0.5, 0.15), (0.9, 0.18)], mcs=1_000_000, n_rec=100,
                   seed=1, init=INIT_FULL)
STREAM_L4M = dict(name="pcpd_L4194304_S1024", L=1 << 22, S=1024, runs=[(0.5, 0.15)],
                  mcs=100_000, n_rec=0, seed=1, init=INIT_FULL)


def batch_instances(n: int = 512, seed: int = 1, l_min_log2: int = 10, l_max_log2: int = 18):
    """Heterogeneous instance mix: L log-uniform in [2^10, 2^18] (rounded to an integer),
    samples in {64, 256, 1024}, d in {.1,.3,.5,.7,.9}, p uniform in [.05,.25], MCS
    log-uniform in [1e3, 1e5] (rounded), full or random-half start by coin, seed 1000+i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        L = int(round(2.0 ** rng.uniform(l_min_log2, l_max_log2)))
        S = int(rng.choice([64, 256, 1024]))
        d = float(rng.choice([0.1, 0.3, 0.5, 0.7, 0.9]))
        p = float(rng.uniform(0.05, 0.25))
        mcs = int(round(10.0 ** rng.uniform(3.0, 5.0)))
        init = INIT_FULL if rng.integers(0, 2) == 0 else INIT_HALF
        out.append(dict(L=L, S=S, p=p, d=d, mcs=mcs, init=init, seed=1000 + i))
    return out


def request_stream(rate_hz: float = 200.0, duration_s: float = 60.0, seed: int = 1,
                   mcs_scale: float = 1.0):
    """Poisson arrivals of simulation requests: L log-uniform in [2^10, 2^20], samples
    log-uniform over powers of two in [64, 4096], p in [.05,.25], d in [.1,.9], MCS
    log-uniform in [1e3, 1e5] times mcs_scale (>= 1)."""
    rng = np.random.default_rng(seed)
    t, out, i = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        L = int(round(2.0 ** rng.uniform(10, 20)))
        S = int(2 ** rng.integers(6, 13))
        p = float(rng.uniform(0.05, 0.25))
        d = float(rng.uniform(0.1, 0.9))
        mcs = max(1, int(round(10.0 ** rng.uniform(3.0, 5.0) * mcs_scale)))
        out.append(dict(arrival=t, L=L, S=S, p=p, d=d, mcs=mcs, init=INIT_FULL, seed=1 + i))
        i += 1
    return out
