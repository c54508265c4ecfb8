"""Pins the Monte Carlo oracles to exactly integrated master equations on tiny rings
(L <= 10), pins those master equations to Eq. (1) and Alg. 1, and pins the random-sequential
oracle to the random dimer-filling (Flory) jamming limit."""
import math

import numpy as np
import pytest

from oracle import exact as E
from paper_1301_6082_gb300.workloads import INIT_FULL, INIT_HALF


def _batch_means(ps: np.ndarray, L: int, batch: int, exact_var=None):
    """Ensemble mean of rho and its standard error from batch means (batches = phase groups,
    whose samples share the random phase).  The error is floored at the exact i.i.d. error
    sqrt(Var[rho]/S) from the master equation, so that a finite ensemble that happens to be
    fully absorbed (zero spread) is not held to a zero error bar."""
    R, S = ps.shape
    g = ps.astype(np.float64).reshape(R, S // batch, batch).mean(2) / L
    se = g.std(1, ddof=1) / math.sqrt(g.shape[1])
    if exact_var is not None:
        se = np.maximum(se, np.sqrt(np.asarray(exact_var) / S))
    return g.mean(1), se


def test_alg1_kernel_reproduces_eq1_rates():
    # One Alg. 1 attempt on the bond of a pair "0AA0" (sites i-1..i+2): the transition
    # probabilities are Eq. (1)'s rates: AA->00 with p(1-d), fission to either side with
    # (1-p)(1-d)/2 each, and the swap (no visible change for AA) with d.
    p, d = 0.17, 0.35
    K = E.bond_kernel_alg1(d, p)
    old = 0b0110
    assert K[0b0000, old] == pytest.approx(p * (1 - d))
    assert K[0b1110, old] == pytest.approx((1 - p) * (1 - d) / 2)
    assert K[0b0111, old] == pytest.approx((1 - p) * (1 - d) / 2)
    assert K[0b0110, old] == pytest.approx(d)
    # "A0" bond: only diffusion acts, with rate d (A0 <-> 0A)
    assert K[0b0010, 0b0100] == pytest.approx(d)
    assert K[0b0100, 0b0100] == pytest.approx(1 - d)
    assert np.allclose(K.sum(0), 1.0)


def test_window_kernel_is_alg1_on_three_site_ring():
    # On L = 3 one window covers the whole ring and its orientation picks one of the three
    # bonds, so a schedule sub-step is one Alg. 1 attempt (fission "low" and "high" land on
    # the same site).  The two are written independently (window form vs Alg. 1 form).
    for p, d in [(0.15, 0.5), (0.3, 0.1), (0.0, 0.0), (1.0, 0.0)]:
        from oracle import oracle as O
        td, tda, tp = O.thresholds(p, d)
        # use exactly equal phase and site laws so that the identity is exact
        w = np.full(3, 1 / 3)
        for x in range(8):
            v = np.zeros(8)
            v[x] = 1
            # window form: P_A = p(1-d) corresponds to Alg. 1's (1-d)*p
            a = E.sched_substep(v, 3, td, tda, phase_w=w)
            tp_equiv = round((tda - td) / (2**32 - td) * 2**32) if td < 2**32 else 0
            b = E.rs_attempt(v, 3, td, tp_equiv, site_w=w)
            np.testing.assert_allclose(a, b, atol=1e-9)


@pytest.mark.parametrize("L", [3, 4, 5, 6, 7, 8, 9, 10])
@pytest.mark.parametrize("p,d", [(0.15, 0.5), (0.3, 0.1)])
def test_schedule_oracle_matches_exact_chain(oracle_mod, L, p, d):
    td, tda, _ = oracle_mod.thresholds(p, d)
    S = 16384
    rec = [1, 2, 4, 8, 16, 32]
    ex, var = E.sched_moments(L, td, tda, rec)
    st = oracle_mod.init_state(L, S, INIT_FULL, 1)
    _, ps, _ = oracle_mod.run(st, p, d, 100 + L, 0, rec[-1], rec, per_sample=True)
    m, se = _batch_means(ps, L, 128, var)    # batch means over phase groups (128 samples)
    assert np.all(np.abs(m - ex) <= 3 * se + 1e-12), (m, ex, se)


@pytest.mark.parametrize("L", [5, 8])
def test_schedule_oracle_random_half_start(oracle_mod, L):
    p, d = 0.2, 0.3
    td, tda, _ = oracle_mod.thresholds(p, d)
    S = 16384
    rec = [0, 3, 9, 27]
    ex, var = E.sched_moments(L, td, tda, rec, mode="half")
    st = oracle_mod.init_state(L, S, INIT_HALF, 17)
    _, ps, _ = oracle_mod.run(st, p, d, 17, 0, rec[-1], rec, per_sample=True)
    m, se = _batch_means(ps, L, 128, var)
    assert np.all(np.abs(m - ex) <= 3 * se + 1e-12), (m, ex, se)


@pytest.mark.parametrize("L", [4, 6, 9])
def test_rs_oracle_matches_exact_chain(oracle_mod, L):
    p, d = 0.15, 0.5
    td, _, tp = oracle_mod.thresholds(p, d)
    S = 2048
    rec = [L * t for t in (1, 2, 5, 10)]
    ex, var = E.rs_moments(L, td, tp, rec)
    st = oracle_mod.init_state(L, S, INIT_FULL, 1)
    _, ps = oracle_mod.rs_run(st, p, d, 3, 0, rec[-1], rec, per_sample=True)
    m, se = _batch_means(ps, L, 32, var)   # RS samples are independent; batches of 32
    assert np.all(np.abs(m - ex) <= 3 * se + 1e-12), (m, ex, se)


def test_rs_dimer_filling_jamming_limit(oracle_mod):
    # d = 0, p = 1 from full: Alg. 1 removes random adjacent pairs until none is left; the
    # remaining density on a large ring tends to exp(-2) (random sequential dimer filling,
    # Flory 1939; the complement of the jammed dimer coverage 1 - e^-2).
    L, S = 4096, 32
    td, _, tp = oracle_mod.thresholds(1.0, 0.0)
    st = oracle_mod.init_state(L, S, INIT_FULL, 1)
    rec = [40 * L]
    tot, ps = oracle_mod.rs_run(st, 1.0, 0.0, 5, 0, rec[-1], rec, per_sample=True)
    rho = ps[0] / L
    # jammed: no adjacent pair is left anywhere
    assert not np.any(st & np.roll(st, -1, axis=1))
    assert abs(rho.mean() - math.exp(-2)) < 4 * rho.std(ddof=1) / math.sqrt(S) + 1.0 / L


def test_pair_occupation_definition():
    # bit i of x is site i; pairs (i, i+1 mod L)
    occ = E.pair_occupation(4)
    assert occ[0b1111] == 4 and occ[0] == 0 and occ[0b0011] == 1 and occ[0b1001] == 1 and occ[0b0101] == 0


@pytest.mark.parametrize("L", [4, 7, 9])
def test_pair_density_matches_exact_chain(oracle_mod, L):
    # the pair density rho_pair = <q_i q_{i+1}> analysed beside rho in Sec. 5.3; batch means
    # over 16 independent seeds (1024 samples each), 3 sigma
    p, d = 0.15, 0.5
    td, tda, _ = oracle_mod.thresholds(p, d)
    rec = [0, 2, 5, 11, 24]
    ex, var = E.sched_observable(L, td, tda, rec, E.pair_occupation(L), mode="half")
    S, means = 1024, []
    for seed in range(40, 56):
        st = oracle_mod.init_state(L, S, INIT_HALF, seed)
        _, _, _, prs = oracle_mod.run(st, p, d, seed, 0, rec[-1], rec, pairs=True)
        means.append(prs.astype(float) / (L * S))
    means = np.array(means)
    m = means.mean(0)
    se = np.maximum(means.std(0, ddof=1) / np.sqrt(len(means)), np.sqrt(var / (S * len(means))))
    assert np.all(np.abs(m - ex) <= 3 * se + 1e-12), (m, ex, se)


def test_pair_counts_closed_forms(oracle_mod):
    for mode, want in ((0, 1.0), (1, 0.0)):
        st = oracle_mod.init_state(30, 64, mode, 1)
        tot, _, _, prs = oracle_mod.run(st, 0.0, 1.0, 1, 0, 5, [0, 5], pairs=True)
        assert np.all(prs == want * 30 * 64)     # full ring: L pairs per sample; empty: none
