"""Pins the threshold reading (Eq. (1) rates as integer thresholds) against exact rational
arithmetic and the special values the definition fixes."""
from fractions import Fraction

import pytest

TWO32 = 1 << 32


@pytest.mark.parametrize("p,d", [(0.15, 0.5), (0.11, 0.1), (0.18, 0.9), (0.0, 0.0), (1.0, 0.0),
                                 (0.0, 1.0), (1.0, 1.0), (0.125141, 0.25), (0.191789, 0.75),
                                 (0.05, 0.3), (0.25, 0.7), (1e-12, 1e-12)])
def test_thresholds_vs_exact_rationals(oracle_mod, p, d):
    td, tda, tp = oracle_mod.thresholds(p, d)
    # d*2^32 is exact in binary floating point, so T_D is the exact floor
    assert td == min(TWO32, int(Fraction(d) * TWO32))
    exact_a = Fraction(p) * (1 - Fraction(d)) * TWO32
    ta = tda - td
    if td + int(exact_a) <= TWO32:
        # two roundings (1-d, p*(1-d)) move the floor by at most one unit
        assert abs(ta - int(exact_a)) <= 1
    assert 0 <= td <= tda <= TWO32
    assert tp == min(TWO32, int(Fraction(p) * TWO32))


def test_threshold_special_values(oracle_mod):
    assert oracle_mod.thresholds(0.3, 0.5)[0] == 1 << 31          # d = 1/2 -> half the range
    assert oracle_mod.thresholds(0.0, 0.25)[:2] == (1 << 30, 1 << 30)  # p = 0: no annihilation
    assert oracle_mod.thresholds(1.0, 0.0)[:2] == (0, TWO32)       # always annihilate
    assert oracle_mod.thresholds(0.7, 1.0)[:2] == (TWO32, TWO32)   # always diffuse
    assert oracle_mod.thresholds(0.5, 0.0)[1] == 1 << 31
    with pytest.raises(ValueError):
        oracle_mod.thresholds(1.5, 0.1)
    with pytest.raises(ValueError):
        oracle_mod.thresholds(float("nan"), 0.1)


def test_substep_of_time(oracle_mod):
    # n_t = ceil(t*L/K), K = floor(L/3); brute force: smallest n with n*K >= t*L
    for L in (3, 4, 5, 8, 10, 1024, 65536, 1 << 22, 1000003):
        K = L // 3
        for t in (0, 1, 2, 3, 7, 100, 2000, 10**6):
            n = oracle_mod.substep_of_time(L, t)
            assert n * K >= t * L and (n == 0 or (n - 1) * K < t * L)
    assert oracle_mod.substep_of_time(1024, 2000) == 6006
    assert oracle_mod.substep_of_time(65536, 10**6) == -(-(10**6 * 65536) // 21845)


def test_phase_is_uniform_law(oracle_mod):
    # phi = floor(x*L/2^32): over many sub-steps each phase of a small ring appears ~1/L
    import numpy as np
    L = 7
    ph = np.array([oracle_mod.phase(3, L, 0, n) for n in range(7000)])
    assert ph.min() == 0 and ph.max() == L - 1
    cnt = np.bincount(ph, minlength=L)
    assert np.all(np.abs(cnt - 1000) < 5 * np.sqrt(1000))
