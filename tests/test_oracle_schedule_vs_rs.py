"""Schedule vs Alg. 1 (random-sequential).  The random-phase window schedule and Alg. 1 are
different Markov chains with the same per-bond marginal rates (Eq. (1)).  These tests pin
the *size* of their difference, measured exactly on tiny rings and by Monte Carlo at the
L = 1024 workload, so that a change in either oracle that moves them apart is caught.
The measured gap is larger than the Monte Carlo error at the L = 1024 workload's own size,
so a plain "agree within 3 sigma" does not hold there; the design notes record the numbers."""
import numpy as np
import pytest

from oracle import exact as E
from paper_1301_6082_gb300.workloads import INIT_FULL, log_times


@pytest.mark.parametrize("L", [6, 8, 9, 10])
def test_exact_gap_small_rings(oracle_mod, L):
    p, d = 0.15, 0.5
    td, tda, tp = oracle_mod.thresholds(p, d)
    ts = [1, 2, 4, 8, 16]
    sub = [oracle_mod.substep_of_time(L, t) for t in ts]
    a = E.sched_density(L, td, tda, sub)
    b = E.rs_density(L, td, tp, [t * L for t in ts])
    gap = a - b
    # measured: the schedule decays faster; |gap| <= 0.025 on these rings
    assert np.all(gap < 0) and np.all(np.abs(gap) <= 0.025), gap


@pytest.mark.slow
def test_gap_at_L1024(oracle_mod):
    p, d, L, S = 0.15, 0.5, 1024, 1024
    ts = [1, 2, 5, 10, 20, 50, 100]
    sub = [oracle_mod.substep_of_time(L, t) for t in ts]
    st = oracle_mod.init_state(L, S, INIT_FULL, 1)
    _, ps, _ = oracle_mod.run(st, p, d, 1, 0, sub[-1], sub, per_sample=True)
    st2 = oracle_mod.init_state(L, S, INIT_FULL, 1)
    _, ps2 = oracle_mod.rs_run(st2, p, d, 1, 0, ts[-1] * L, [t * L for t in ts], per_sample=True)
    a = ps.astype(float).mean(1) / L
    b = ps2.astype(float).mean(1) / L
    rel = a / b - 1
    # same trend as the exact small-ring chains: the schedule is below Alg. 1, by at most
    # ~5% at t = 1 MCS and by 1-4% afterwards
    assert np.all(rel < 0.005) and np.all(rel > -0.06), rel
    assert rel[0] < -0.02          # the early transient differs clearly
    assert np.all(np.abs(rel[3:]) < 0.045), rel
