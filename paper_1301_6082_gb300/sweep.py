"""Near-critical sweeps (Sec. 5.3): several annihilation rates p at one diffusion rate d,
each with several independent seeds, run as one batch on the GPU; returns the particle and
pair densities at log-spaced times and their effective exponents.  Over several GPUs, each
rank runs a group range of every (p, seed) ensemble (paper_1301_6082_gb300.replicas) and the
ranks sum their counts exactly."""
from __future__ import annotations

import numpy as np

from . import pcpd
from .analysis import effective_exponent, jackknife_effective_exponent
from .workloads import INIT_FULL, log_times


def p_sweep(d: float, ps, L: int, samples: int, mcs: int, n_rec: int = 60, seeds=(1,),
            init: int = INIT_FULL, tuple_n: int = 2):
    """Run every (p, seed) pair for `mcs` MCS from a full lattice in one batch (tuple_n = 3 /
    4: the TCPD / QCPD).  Returns a dict p -> {"t", "rho", "rho_pair", "delta_eff",
    "delta_eff_pair"} with densities averaged over the seeds (counts summed exactly before
    dividing); with two or more seeds also "rho_err", "rho_pair_err", "delta_eff_err" and
    "delta_eff_pair_err", jackknife standard errors over the seeds (independent replicas)."""
    times = log_times(mcs, n_rec)
    b = pcpd.Batch()
    index = []
    for p in ps:
        for s in seeds:
            index.append((p, b.add(L, samples, p, d, s, mcs, times, init=init, tuple_n=tuple_n)))
    b.run()
    out = {}
    for p in ps:
        ids = [i for (q, i) in index if q == p]
        tot = sum(b.counts(i).astype(np.int64) for i in ids)
        prs = sum(b.pair_counts(i).astype(np.int64) for i in ids)
        denom = float(L) * samples * len(ids)
        rho, rho_pair = tot / denom, prs / denom
        _, rm, de = effective_exponent(times, rho)
        _, rpm, dep = effective_exponent(times, rho_pair)
        out[p] = {"t": np.array(times), "rho": rho, "rho_pair": rho_pair,
                  "delta_eff": (rm, de), "delta_eff_pair": (rpm, dep)}
        if len(ids) >= 2:
            norm = float(L) * samples
            per = np.array([b.counts(i) for i in ids], dtype=np.float64) / norm
            per_pair = np.array([b.pair_counts(i) for i in ids], dtype=np.float64) / norm
            try:
                _, out[p]["rho_err"], _, _, out[p]["delta_eff_err"] = jackknife_effective_exponent(times, per)
                _, out[p]["rho_pair_err"], _, _, out[p]["delta_eff_pair_err"] = \
                    jackknife_effective_exponent(times, per_pair)
            except ValueError:   # a replica died out: no error bars for this p
                pass
    b.close()
    return out
