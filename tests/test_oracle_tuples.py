"""Pins of the oracle for the n-tuple processes (TCPD n = 3, QCPD n = 4; R14): invariants,
closed forms and the exact schedule chain on tiny rings."""
import math

import numpy as np
import pytest

from oracle import exact as E
from paper_1301_6082_gb300.workloads import INIT_EMPTY, INIT_FULL, INIT_HALF

TUPLES = [3, 4]


def test_tuple_kernel_at_n2_is_the_pcpd_window_kernel():
    # two independent formulations of the 3-site window (R2 and R14 at n = 2)
    for pD, pA in ((0.5, 0.075), (0.1, 0.3), (0.0, 1.0), (1.0, 0.0)):
        np.testing.assert_allclose(E.tuple_window_kernel(pD, pA, 2), E.window_kernel(pD, pA), atol=1e-15)


@pytest.mark.parametrize("n", TUPLES)
def test_tuple_kernel_is_stochastic_and_conserving_where_it_must(n):
    K = E.tuple_window_kernel(0.3, 0.2, n)
    np.testing.assert_allclose(K.sum(0), 1.0, atol=1e-14)
    W = n + 1
    # empty window stays empty; a window with no full tuple only diffuses (N conserved)
    assert K[0, 0] == pytest.approx(1.0)
    for old in range(1 << W):
        bits = [(old >> (W - 1 - j)) & 1 for j in range(W)]
        full0, full1 = all(bits[:n]), all(bits[1:])
        if not (full0 or full1):
            for new in np.flatnonzero(K[:, old]):
                assert bin(int(new)).count("1") == sum(bits)


@pytest.mark.parametrize("n", TUPLES)
def test_empty_stays_empty(oracle_mod, n):
    st = oracle_mod.init_state(40, 64, INIT_EMPTY, 1)
    tot, _, ev = oracle_mod.run(st, 0.2, 0.4, 3, 0, 50, [50], tuple_n=n)
    assert tot[0] == 0 and st.sum() == 0 and ev[1] == 0 and ev[2] == 0


@pytest.mark.parametrize("n", TUPLES)
def test_bookkeeping_and_d1_conservation(oracle_mod, n):
    L, S = 97, 64
    st = oracle_mod.init_state(L, S, INIT_HALF, 5)
    n0 = int(st.sum())
    tot, _, ev = oracle_mod.run(st, 0.1, 0.3, 9, 0, 150, [0, 150], tuple_n=n)
    assert tot[0] == n0
    assert int(tot[1]) == n0 + int(ev[2]) - n * int(ev[1])   # each window: +1, -n or 0
    assert ev[1] > 0 and ev[2] > 0 and ev[0] > 0
    st = oracle_mod.init_state(L, S, INIT_HALF, 6)
    before = st.sum(1)
    _, ps, ev = oracle_mod.run(st, 0.4, 1.0, 4, 0, 60, [60], per_sample=True, tuple_n=n)
    np.testing.assert_array_equal(ps[0], before)
    assert ev[1] == 0 and ev[2] == 0


@pytest.mark.parametrize("n", TUPLES)
@pytest.mark.parametrize("L", [60, 61, 64])
def test_p1_d0_first_substep_closed_form(oracle_mod, n, L):
    # every window's tuple is full at the start and annihilates: N = L - n*floor(L/(n+1))
    st = oracle_mod.init_state(L, 64, INIT_FULL, 1)
    _, ps, _ = oracle_mod.run(st, 1.0, 0.0, 2, 0, 1, [1], per_sample=True, tuple_n=n)
    assert np.all(ps[0] == L - n * (L // (n + 1)))


@pytest.mark.parametrize("n", TUPLES)
def test_full_lattice_first_substep_binomial(oracle_mod, n):
    L, S, p, d = 300, 2048, 0.15, 0.5
    td, tda, _ = oracle_mod.thresholds(p, d)
    pa = (tda - td) / 2**32
    K = L // (n + 1)
    st = oracle_mod.init_state(L, S, INIT_FULL, 1)
    _, ps, _ = oracle_mod.run(st, p, d, 21, 0, 1, [1], per_sample=True, tuple_n=n)
    m = L - ps[0].astype(np.int64)
    assert np.all(m % n == 0)
    a = m // n
    assert abs(a.mean() - K * pa) < 4 * math.sqrt(K * pa * (1 - pa) / S)
    assert abs(a.var(ddof=1) / (K * pa * (1 - pa)) - 1) < 4 * math.sqrt(2 / (S - 1))


@pytest.mark.parametrize("n", TUPLES)
def test_substep_of_time_is_least_cover(oracle_mod, n):
    for L in (n + 1, 10, 97, 1024, 65536):
        K = L // (n + 1)
        for t in (0, 1, 2, 7, 1000):
            ns = oracle_mod.substep_of_time(L, t, n)
            assert ns * K >= t * L and (ns == 0 or (ns - 1) * K < t * L)


def _batch_means(ps, L, bs, var):
    x = ps.astype(np.float64) / L
    S = x.shape[1]
    nb = S // bs
    bm = x[:, : nb * bs].reshape(x.shape[0], nb, bs).mean(2)
    m = bm.mean(1)
    se = bm.std(1, ddof=1) / math.sqrt(nb)
    return m, np.maximum(se, np.sqrt(var / S))


@pytest.mark.parametrize("n,L", [(3, 4), (3, 5), (3, 7), (3, 9), (4, 5), (4, 6), (4, 8), (4, 10)])
def test_schedule_oracle_matches_exact_chain(oracle_mod, n, L):
    p, d = 0.15, 0.5
    td, tda, _ = oracle_mod.thresholds(p, d)
    S = 16384
    rec = [1, 2, 4, 8, 16, 32]
    ex, var = E.sched_moments(L, td, tda, rec, tuple_n=n)
    st = oracle_mod.init_state(L, S, INIT_FULL, 1)
    _, ps, _ = oracle_mod.run(st, p, d, 300 + L, 0, rec[-1], rec, per_sample=True, tuple_n=n)
    m, se = _batch_means(ps, L, 128, var)    # batch means over phase groups (128 samples)
    assert np.all(np.abs(m - ex) <= 3 * se + 1e-12), (m, ex, se)


def test_tuple_two_is_the_pcpd(oracle_mod):
    a = oracle_mod.init_state(50, 64, INIT_HALF, 4)
    b = a.copy()
    ta, _, _ = oracle_mod.run(a, 0.2, 0.4, 6, 0, 30, [30])
    tb, _, _ = oracle_mod.run(b, 0.2, 0.4, 6, 0, 30, [30], tuple_n=2)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ta, tb)


def test_bad_tuple_sizes_are_refused(oracle_mod):
    st = oracle_mod.init_state(10, 32, INIT_FULL, 1)
    for n in (1, 5):
        with pytest.raises(ValueError):
            oracle_mod.run(st, 0.2, 0.4, 6, 0, 3, tuple_n=n)
    small = oracle_mod.init_state(4, 32, INIT_FULL, 1)
    with pytest.raises(ValueError):
        oracle_mod.run(small, 0.2, 0.4, 6, 0, 3, tuple_n=4)   # L < n + 1
