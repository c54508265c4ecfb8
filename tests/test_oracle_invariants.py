"""Pins of the window-schedule oracle by invariants and closed forms that the method fixes:
absorbing empty state, particle-number changes per event, conservation at d=1, and the
exactly solvable first sub-step from a full lattice."""
import math

import numpy as np
import pytest

from paper_1301_6082_gb300.workloads import INIT_EMPTY, INIT_FULL, INIT_HALF


def test_empty_stays_empty(oracle_mod):
    # The empty lattice is the absorbing state of the PCPD (Sec. 1-2).
    st = oracle_mod.init_state(64, 64, INIT_EMPTY, 1)
    tot, _, ev = oracle_mod.run(st, 0.15, 0.5, 1, 0, 200, [0, 50, 200])
    assert tot.tolist() == [0, 0, 0] and st.sum() == 0 and ev.tolist() == [0, 0, 0]


@pytest.mark.parametrize("p,d", [(0.15, 0.5), (0.05, 0.1), (0.3, 0.9)])
def test_particle_number_bookkeeping(oracle_mod, p, d):
    # Each window event changes N by +1 (fission into an empty site), -2 (annihilation) or 0;
    # the oracle asserts this per window, and the totals must reconcile with the event counts.
    L, S = 97, 64
    st = oracle_mod.init_state(L, S, INIT_HALF, 5)
    n0 = int(st.sum())
    tot, _, ev = oracle_mod.run(st, p, d, 9, 0, 120, [0, 120])
    assert tot[0] == n0
    assert int(tot[1]) == n0 + int(ev[2]) - 2 * int(ev[1])
    assert ev[1] > 0 and ev[2] > 0 and (d == 0 or ev[0] > 0)


@pytest.mark.parametrize("L", [10, 64, 101])
def test_d1_conserves_particles_per_sample(oracle_mod, L):
    st = oracle_mod.init_state(L, 64, INIT_HALF, 3)
    before = st.sum(1)
    _, ps, ev = oracle_mod.run(st, 0.4, 1.0, 4, 0, 90, [90], per_sample=True)
    np.testing.assert_array_equal(ps[0], before)
    assert ev[0] > 0 and ev[1] == 0 and ev[2] == 0   # particles did move, nothing reacted
    assert not np.array_equal(st, oracle_mod.init_state(L, 64, INIT_HALF, 3))


@pytest.mark.parametrize("p,d", [(0.0, 0.3), (0.2, 1.0)])
def test_full_lattice_stays_full(oracle_mod, p, d):
    # p = 0: no annihilation, fission into occupied sites is a no-op; d = 1: swaps of ones.
    st = oracle_mod.init_state(50, 64, INIT_FULL, 1)
    tot, _, _ = oracle_mod.run(st, p, d, 2, 0, 60, [60])
    assert tot[0] == 50 * 64


def test_p1_d0_first_substep_closed_form(oracle_mod):
    # p=1, d=0 from full: every window annihilates its bond -> rho = 1 - 2K/L exactly.
    for L in (8, 1024, 1025):
        st = oracle_mod.init_state(L, 64, INIT_FULL, 1)
        _, ps, _ = oracle_mod.run(st, 1.0, 0.0, 11, 0, 1, [1], per_sample=True)
        assert np.all(ps[0] == L - 2 * (L // 3))
    assert (1024 - 2 * 341) / 1024 == 1 - 682 / 1024


@pytest.mark.parametrize("p,d", [(0.15, 0.5), (0.6, 0.2)])
def test_full_lattice_first_substep_binomial(oracle_mod, p, d):
    # From full, one sub-step: each of the K windows annihilates independently with
    # probability P_A = (T_DA - T_D)/2^32, so N = L - 2*Binomial(K, P_A) per sample.
    L, S = 300, 2048
    td, tda, _ = oracle_mod.thresholds(p, d)
    pa = (tda - td) / 2**32
    K = L // 3
    st = oracle_mod.init_state(L, S, INIT_FULL, 1)
    _, ps, _ = oracle_mod.run(st, p, d, 21, 0, 1, [1], per_sample=True)
    m = (L - ps[0].astype(np.int64))
    assert np.all(m % 2 == 0)
    a = m // 2
    assert abs(a.mean() - K * pa) < 4 * math.sqrt(K * pa * (1 - pa) / S)
    assert abs(a.var(ddof=1) / (K * pa * (1 - pa)) - 1) < 4 * math.sqrt(2 / (S - 1))


def test_run_splits_compose(oracle_mod):
    # Counter-based randomness: running [0, 40) then [40, 90) equals running [0, 90).
    L, S = 40, 64
    a = oracle_mod.init_state(L, S, INIT_HALF, 8)
    b = a.copy()
    oracle_mod.run(a, 0.2, 0.4, 6, 0, 90)
    oracle_mod.run(b, 0.2, 0.4, 6, 0, 40)
    oracle_mod.run(b, 0.2, 0.4, 6, 40, 90)
    np.testing.assert_array_equal(a, b)


def test_pack_roundtrip(oracle_mod):
    st = oracle_mod.init_state(33, 96, INIT_HALF, 2)
    w = oracle_mod.pack(st)
    assert w.shape == (3, 33) and w.dtype == np.uint32
    np.testing.assert_array_equal(oracle_mod.unpack(w), st)
    # random-half init: bit j of group g's word at site i is the INIT Philox word's bit j
    ctr = np.array([[i, 0, g, 2 << 28] for g in range(3) for i in range(33)], dtype=np.uint32)
    np.testing.assert_array_equal(w.reshape(-1), oracle_mod.philox(ctr, 2)[:, 0])


def test_oracle_still_writes_the_stored_golden_run(oracle_mod):
    """Regression guard for refactors of the oracle: the stored L=1024, 64-sample decay run
    (written by tests/golden/make_golden.py from an earlier oracle) is reproduced."""
    import os
    from paper_1301_6082_gb300.workloads import SMALL_L1024, log_times
    w = SMALL_L1024
    L, S = w["L"], w["S"]
    d, p = w["runs"][0]
    ts = log_times(w["mcs"], w["n_rec"])
    sub = [oracle_mod.substep_of_time(L, t) for t in ts]
    st = oracle_mod.init_state(L, S, w["init"], w["seed"])
    tot, _, _ = oracle_mod.run(st, p, d, w["seed"], 0, sub[-1], sub)
    golden = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "pcpd_L1024_S64.txt"), dtype=np.uint64)
    np.testing.assert_array_equal(golden[:, 1], np.array(sub, dtype=np.uint64))
    np.testing.assert_array_equal(golden[:, 2], tot)
