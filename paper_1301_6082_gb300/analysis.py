"""Host-side analysis of recorded densities (Sec. 5.3): the effective decay exponent
delta_eff between consecutive records, -d ln rho / d ln t, which the paper plots against the
density itself for both the particle density and the pair density."""
from __future__ import annotations

import numpy as np


def effective_exponent(times, rho):
    """delta_eff on each interval between consecutive records with t > 0 and rho > 0:
    -(ln rho[k+1] - ln rho[k]) / (ln t[k+1] - ln t[k]).  Returns (t_mid, rho_mid, delta),
    with the geometric means of the interval's end points as t_mid and rho_mid."""
    t = np.asarray(times, dtype=np.float64)
    r = np.asarray(rho, dtype=np.float64)
    keep = (t > 0) & (r > 0)
    t, r = t[keep], r[keep]
    lt, lr = np.log(t), np.log(r)
    delta = -(lr[1:] - lr[:-1]) / (lt[1:] - lt[:-1])
    return np.exp(0.5 * (lt[1:] + lt[:-1])), np.exp(0.5 * (lr[1:] + lr[:-1])), delta


def jackknife_effective_exponent(times, rho_replicas):
    """Mean density over independent replicas (seeds, or 128-sample phase groups) with
    jackknife standard errors, and delta_eff of the mean with jackknife errors.

    rho_replicas: [R][T] densities of R >= 2 independent replicas at the record times.
    Returns (rho_mean, rho_err, t_mid, delta, delta_err); delta is effective_exponent of the
    mean.  The jackknife recomputes delta_eff with each replica left out in turn:
    err^2 = (R-1)/R * sum_j (delta_(j) - mean_j delta_(j))^2."""
    x = np.asarray(rho_replicas, dtype=np.float64)
    if x.ndim != 2 or x.shape[0] < 2:
        raise ValueError("need at least two replicas")
    R = x.shape[0]
    mean = x.mean(0)
    loo = (x.sum(0)[None, :] - x) / (R - 1)          # leave-one-out means
    rho_err = np.sqrt((R - 1) / R * ((loo - loo.mean(0)) ** 2).sum(0))
    tm, _, delta = effective_exponent(times, mean)
    deltas = np.array([effective_exponent(times, row)[2] for row in loo])
    if deltas.shape[1] != delta.shape[0]:
        raise ValueError("a leave-one-out mean has non-positive entries where the mean has none")
    delta_err = np.sqrt((R - 1) / R * ((deltas - deltas.mean(0)) ** 2).sum(0))
    return mean, rho_err, tm, delta, delta_err


PHASE_GROUP = 128   # samples that share the random window phase of every sub-step


def phase_group_densities(sample_counts, L: int):
    """Densities of each 128-sample phase group at every record: the independent replicas of
    one run.  Samples of a phase group share the window phase of every sub-step and so are
    correlated; distinct phase groups are independent, so error bars take batch means over
    them (feed the result to jackknife_effective_exponent).

    sample_counts: [R][S] occupied sites per sample at R records (S a multiple of 128).
    Returns [S/128][R] densities."""
    c = np.asarray(sample_counts, dtype=np.float64)
    if c.ndim != 2 or c.shape[1] % PHASE_GROUP:
        raise ValueError("need [records][samples] counts with samples a multiple of 128")
    R, S = c.shape
    return c.reshape(R, S // PHASE_GROUP, PHASE_GROUP).sum(axis=2).T / (PHASE_GROUP * float(L))
