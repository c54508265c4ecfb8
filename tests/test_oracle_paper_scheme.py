"""Pins of the oracle's version of the paper's own GPU scheme (Sec. 3-4, Alg. 2): one
shared random local site per step, connected-lattice multispin words, dyadic diffusion
masks, decorrelation words ANDed with a broadcast annihilation draw."""
import math

import numpy as np
import pytest


def test_empty_stays_empty(oracle_mod):
    st = np.zeros((2, 32 * 4 * 32), np.uint8)
    tot = oracle_mod.paper_run(st, 4, 32, 0.2, 0.5, 1, 2, 1, 0, 30, [30])
    assert tot[0] == 0 and st.sum() == 0


def test_d1_conserves(oracle_mod):
    rng = np.random.default_rng(1)
    st = (rng.random((3, 32 * 5 * 32)) < 0.5).astype(np.uint8)
    n0 = st.sum(1)
    oracle_mod.paper_run(st, 5, 32, 0.2, 1.0, 1, 2, 3, 0, 25)
    np.testing.assert_array_equal(st.sum(1), n0)


@pytest.mark.parametrize("n_loc,S_w", [(4, 32), (6, 64), (9, 32)])
def test_same_local_site_in_every_workitem(oracle_mod, n_loc, S_w):
    # d = 0, p = 1, no decorrelation: one step from full annihilates exactly the bonds at the
    # shared local site of every (bit, workitem) segment: 32*S_w bonds spaced n_loc apart
    L = 32 * n_loc * S_w
    st = np.ones((4, L), np.uint8)
    tot = oracle_mod.paper_run(st, n_loc, S_w, 1.0, 0.0, 1, 0, 11, 0, 1, [1])
    assert tot[0] == 4 * (L - 2 * 32 * S_w)
    for row in st:
        empty = np.flatnonzero(row == 0)
        assert len(empty) == 2 * 32 * S_w
        r = sorted(set((empty % n_loc).tolist()))
        assert len(r) == 2 and (r[1] - r[0]) % n_loc in (1, n_loc - 1)


@pytest.mark.parametrize("p,n_dec", [(0.15, 2), (0.3, 1), (0.1, 0)])
def test_first_step_annihilation_law(oracle_mod, p, n_dec):
    # From full, d = 1/2: in each workitem the number of annihilated bonds is C * B with
    # C ~ Bernoulli(T_c/2^32) (one broadcast draw) and B ~ Binomial(32, (1/2) 2^-n_dec);
    # exact mean and variance of the removed particles over many workitems.
    n_loc, S_w, systems = 4, 64, 64
    L = 32 * n_loc * S_w
    _, tc = oracle_mod.paper_thresholds(p, 0.5, 1, n_dec)
    q = tc / 2**32
    pb = 0.5 * 2.0 ** -n_dec
    st = np.ones((systems, L), np.uint8)
    oracle_mod.paper_run(st, n_loc, S_w, p, 0.5, 1, n_dec, 5, 0, 1)
    removed = (L - st.sum(1)) // 2                       # per system: sum over S_w workitems
    mean = S_w * q * 32 * pb
    var_w = q * (32 * pb * (1 - pb) + (32 * pb) ** 2) - (q * 32 * pb) ** 2
    var = S_w * var_w
    m = removed.mean()
    assert abs(m - mean) < 4 * math.sqrt(var / systems), (m, mean)
    v = removed.var(ddof=1)
    assert abs(v / var - 1) < 4 * math.sqrt(2 / (systems - 1)) + 0.05, (v, var)


def test_paper_thresholds_checks(oracle_mod):
    assert oracle_mod.paper_thresholds(0.15, 0.5, 1, 2) == (1, int(0.6 * 2**32))
    assert oracle_mod.paper_thresholds(0.25, 0.75, 2, 2) == (3, 1 << 32)
    with pytest.raises(ValueError):
        oracle_mod.paper_thresholds(0.3, 0.5, 1, 2)     # p * 4 > 1
    with pytest.raises(ValueError):
        oracle_mod.paper_thresholds(0.1, 0.3, 2, 0)     # 0.3 is not a multiple of 1/4


def test_system_offset_and_per_system_counts(oracle_mod):
    # systems are independent streams: running them together equals running each at its offset
    rng = np.random.default_rng(3)
    st = (rng.random((4, 32 * 4 * 32)) < 0.6).astype(np.uint8)
    parts = st.copy()
    tot, ps = oracle_mod.paper_run(st, 4, 32, 0.2, 0.5, 1, 2, 9, 5, 60, [5, 30, 60], per_system=True)
    for s in range(4):
        one = np.ascontiguousarray(parts[s:s + 1])
        t1 = oracle_mod.paper_run(one, 4, 32, 0.2, 0.5, 1, 2, 9, 5, 60, [5, 30, 60], sys0=s)
        np.testing.assert_array_equal(one[0], st[s])
        np.testing.assert_array_equal(t1, ps[:, s])
    np.testing.assert_array_equal(ps.sum(1), tot)
    np.testing.assert_array_equal(ps[-1], st.sum(1))


@pytest.mark.parametrize("d,m", [(0.25, 2), (0.75, 2), (0.375, 3), (0.5, 1)])
def test_one_step_diffusion_law(oracle_mod, d, m):
    # Alternating occupation (no two neighbours occupied): no reaction can happen, and every
    # updated bond holds one particle, so one step moves exactly one particle per diffusing
    # bond: the changed sites are 2 x Binomial(32*S_w*systems, d) -- the dyadic diffusion draw
    # of m planes against T_d = d*2^m.
    n_loc, S_w, systems = 4, 64, 64
    L = 32 * n_loc * S_w
    st = np.zeros((systems, L), np.uint8)
    st[:, 0::2] = 1
    before = st.copy()
    oracle_mod.paper_run(st, n_loc, S_w, 0.1, d, m, 1, 17, 0, 1)
    changed = (st != before).sum(1)
    assert np.all(changed % 2 == 0) and np.array_equal(st.sum(1), before.sum(1))
    swaps = changed // 2
    n = 32 * S_w
    assert abs(swaps.mean() - n * d) < 4 * math.sqrt(n * d * (1 - d) / systems)
    assert abs(swaps.var(ddof=1) / (n * d * (1 - d)) - 1) < 4 * math.sqrt(2 / (systems - 1)) + 0.05


def test_one_step_fission_sides(oracle_mod):
    # Isolated pairs on sites 4k+1, 4k+2 (n_loc a multiple of 4, so a bond's start has the
    # residue of l*), d = 0 and T_c = 0 (no annihilation): a system whose l* hits the pairs
    # (l* = 1 mod 4) puts one particle on 4k or 4k+3 for every bond, left or right with
    # probability 1/2 each; any other l* changes nothing.
    n_loc, S_w, systems = 8, 64, 256
    L = 32 * n_loc * S_w
    st = np.zeros((systems, L), np.uint8)
    st[:, 1::4] = 1
    st[:, 2::4] = 1
    before = st.copy()
    oracle_mod.paper_run(st, n_loc, S_w, 0.0, 0.0, 1, 0, 23, 0, 1)
    added = st.sum(1).astype(np.int64) - before.sum(1)
    hit = added > 0
    assert 0 < hit.sum() < systems
    assert np.all(added[hit] == 32 * S_w) and np.all(added[~hit] == 0)
    left = (st[hit][:, 0::4] == 1).sum(1)
    n = 32 * S_w
    assert abs(left.mean() - n / 2) < 4 * math.sqrt(n / 4 / hit.sum())
