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
