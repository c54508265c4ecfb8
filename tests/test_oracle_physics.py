"""Qualitative physics of the oracle's dynamics (no exact reference at these sizes): the paper
finds p_c < 1/4 at d = 1/2 (Sec. 4.3), so at p = 1/4 the density must keep decaying, while
deep in the active phase (p = 0.01) it settles at a finite value."""
import numpy as np

from paper_1301_6082_gb300.analysis import effective_exponent
from paper_1301_6082_gb300.workloads import INIT_FULL, log_times


def run_density(oracle_mod, L, S, p, d, mcs, n_rec, seed):
    times = log_times(mcs, n_rec)
    subs = [oracle_mod.substep_of_time(L, t) for t in times]
    st = oracle_mod.init_state(L, S, INIT_FULL, seed)
    tot, _, _ = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs)
    return np.array(times, dtype=float), tot / (L * S)


def test_subcritical_decay_and_active_steady_state(oracle_mod):
    L, S, d, mcs = 512, 64, 0.5, 3000
    t, sub = run_density(oracle_mod, L, S, 0.25, d, mcs, 10, seed=4)
    _, act = run_density(oracle_mod, L, S, 0.01, d, mcs, 10, seed=5)
    assert np.all(np.diff(sub) < 0) and sub[-1] < 0.03, sub
    _, _, delta = effective_exponent(t, sub)
    assert delta[-1] > 0.25, delta          # faster than the critical decay (~0.2)
    assert act[-1] > 0.05, act              # a finite active density
    assert abs(act[-1] - act[-2]) < 0.1 * act[-1], act
