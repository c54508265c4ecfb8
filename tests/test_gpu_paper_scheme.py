"""GPU parity of the paper's own scheme (Sec. 3-4, Alg. 2) against the oracle, bit for bit:
record totals, per-system counts and final lattices."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def words_to_sites(words, n_loc, S_w):
    """[systems][n_loc][S_w] words -> [systems][L] bytes; bit b of [l][w] is site
    b*(L/32) + w*n_loc + l."""
    words = np.asarray(words, dtype=np.uint32)
    n = words.shape[0]
    bits = (words[..., None] >> np.arange(32, dtype=np.uint32)) & 1       # [s][l][w][b]
    return np.ascontiguousarray(bits.transpose(0, 3, 2, 1).reshape(n, 32 * n_loc * S_w)).astype(np.uint8)


def sites_to_words(state, n_loc, S_w):
    n = state.shape[0]
    bits = state.reshape(n, 32, S_w, n_loc).transpose(0, 3, 2, 1).astype(np.uint32)  # [s][l][w][b]
    return (bits << np.arange(32, dtype=np.uint32)).sum(-1, dtype=np.uint64).astype(np.uint32)


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1301_6082_gb300 import build, pcpd
    build.build()
    pcpd.load()
    return pcpd


def test_layout_helpers_roundtrip():
    rng = np.random.default_rng(0)
    st = (rng.random((2, 32 * 5 * 64)) < 0.5).astype(np.uint8)
    w = sites_to_words(st, 5, 64)
    np.testing.assert_array_equal(words_to_sites(w, 5, 64), st)
    # site 1 of a system lies in bit 0 of word (l=1, w=0); site L/32 in bit 1 of (0, 0)
    one = np.zeros((1, 32 * 5 * 64), np.uint8)
    one[0, 1] = 1
    one[0, 5 * 64] = 1
    w = sites_to_words(one, 5, 64)
    assert w[0, 1, 0] == 1 and w[0, 0, 0] == 2 and w.sum() == 3


# n_loc, S_w, systems, p, d, m, n_dec, step0, steps, generic
CASES = [
    (4, 32, 3, 0.15, 0.5, 1, 2, 0, 600, False),
    (5, 64, 5, 0.2, 0.25, 2, 2, 17, 500, False),
    (32, 64, 3, 0.15, 0.5, 1, 2, 0, 256, False),      # the paper's L = 65536 layout
    (7, 96, 4, 0.3, 0.75, 2, 1, 3, 300, False),
    (6, 32, 9, 0.05, 0.375, 3, 3, 0, 400, False),     # 9 systems: ragged last CTA
    (4, 128, 2, 0.5, 0.5, 4, 1, 0, 300, False),       # m = 4: runtime-count kernel
    (9, 32, 3, 0.01, 0.5, 1, 5, 0, 200, False),       # n_dec = 5: runtime-count kernel
    (5, 64, 3, 0.15, 0.5, 1, 2, 40, 300, True),       # generic kernel forced
    (4, 32, 2, 0.25, 1.0, 1, 2, 0, 100, False),       # d = 1: every bond swaps
    (4, 32, 2, 0.25, 0.0, 1, 2, 0, 200, False),       # d = 0, p*4 = 1: broadcast draw always passes
    (4, 32, 3, 0.0, 0.5, 1, 0, 0, 150, False),        # p = 0: no annihilation
    (4, 1024, 1, 0.15, 0.5, 1, 2, 0, 60, False),      # S_w = 1024
    (8, 256, 3, 0.15, 0.5, 1, 2, 0, 120, False),      # one system per CTA
    (5, 32, 3, 2.0 ** -9, 37 / 256, 8, 8, 11, 90, False),   # 8 planes, 8 decorrelation words
    (4, 32, 2, 0.5, 1.0, 0, 1, 0, 60, False),         # m = 0: d in {0, 1}
]


@pytest.mark.parametrize("case", CASES, ids=[f"nloc{c[0]}_Sw{c[1]}_n{c[2]}_m{c[5]}_dec{c[6]}{'_gen' if c[9] else ''}"
                                             for c in CASES])
def test_paper_scheme_parity(P, oracle_mod, case):
    n_loc, S_w, systems, p, d, m, n_dec, step0, steps, generic = case
    L = 32 * n_loc * S_w
    rng = np.random.default_rng(n_loc * 1000 + S_w + systems)
    st = (rng.random((systems, L)) < 0.7).astype(np.uint8)
    recs = sorted({step0, step0 + 1, step0 + steps // 3, step0 + steps - 1, step0 + steps})
    seed = 0x1234_5678_9ABC + n_loc
    with P.PaperScheme(n_loc, S_w, systems, p, d, m, n_dec, seed=seed, generic=generic) as h:
        h.set_lattice(sites_to_words(st, n_loc, S_w), step0)
        h.run(steps, recs)
        tot, ps = h.counts(per_system=True)
        lat = words_to_sites(h.lattice(), n_loc, S_w)
        assert h.step == step0 + steps
    ref = st.copy()
    rt, rps = oracle_mod.paper_run(ref, n_loc, S_w, p, d, m, n_dec, seed, step0, step0 + steps, recs,
                                   per_system=True)
    np.testing.assert_array_equal(tot, rt)
    np.testing.assert_array_equal(ps, rps)
    np.testing.assert_array_equal(lat, ref)


def test_paper_scheme_splice_and_resume(P, oracle_mod):
    n_loc, S_w, systems = 6, 64, 4
    args = (0.15, 0.5, 1, 2)
    with P.PaperScheme(n_loc, S_w, systems, *args, seed=7) as a:
        a.run(250, [0, 100, 250])
        ta = a.counts()
        la = a.lattice()
    with P.PaperScheme(n_loc, S_w, systems, *args, seed=7) as b:
        b.run(100, [0, 100])
        mid = b.lattice()
        b.run(150, [250])
        np.testing.assert_array_equal(b.counts(), ta)
        np.testing.assert_array_equal(b.lattice(), la)
        b.set_lattice(mid, 100)
        b.run(150, [100, 250])
        np.testing.assert_array_equal(b.counts(), ta[1:])
        np.testing.assert_array_equal(b.lattice(), la)
    full = np.ones((systems, 32 * n_loc * S_w), np.uint8)
    rt = oracle_mod.paper_run(full, n_loc, S_w, *args, 7, 0, 250, [0, 100, 250])
    np.testing.assert_array_equal(ta, rt)


def test_paper_scheme_systems_per_cta_invariance(P):
    outs = []
    for spc in (1, 2, 3):
        with P.PaperScheme(5, 64, 7, 0.15, 0.5, 1, 2, seed=3, plan_spc=spc) as h:
            assert h.plan()["systems_per_cta"] == spc
            h.run(200, [200])
            outs.append((h.counts(per_system=True)[1], h.lattice()))
    for c, lat in outs[1:]:
        np.testing.assert_array_equal(c, outs[0][0])
        np.testing.assert_array_equal(lat, outs[0][1])


@pytest.mark.parametrize("n_loc,S_w,systems", [(32, 64, 4096), (32, 64, 3648), (64, 32, 3648)])
def test_paper_scheme_full_size_sampled(P, oracle_mod, n_loc, S_w, systems):
    """The bench layouts (L = 65536 as S_w = 64 x n_loc = 32 and S_w = 32 x n_loc = 64; 3648
    systems as the bench runs them, and 4096) from full: sampled systems against the oracle
    run at their system offsets."""
    steps = 100 * n_loc
    args = (0.15, 0.5, 1, 2)
    recs = [0, n_loc, 5 * n_loc, 10 * n_loc, steps]
    with P.PaperScheme(n_loc, S_w, systems, *args, seed=1) as h:
        h.run(steps, recs)
        tot, ps = h.counts(per_system=True)
        lat = h.lattice()
    assert np.array_equal(ps.sum(1, dtype=np.uint64), tot)
    for s in (0, 1, systems // 2, systems - 1):
        ref = np.ones((1, 32 * n_loc * S_w), np.uint8)
        rt = oracle_mod.paper_run(ref, n_loc, S_w, *args, 1, 0, steps, recs, sys0=s)
        np.testing.assert_array_equal(ps[:, s], rt)
        np.testing.assert_array_equal(words_to_sites(lat[s:s + 1], n_loc, S_w), ref)


def test_paper_scheme_bad_args(P):
    bad = [dict(n_loc=3), dict(S_w=48), dict(S_w=2048), dict(systems=0), dict(d=0.3),
           dict(p=0.3), dict(m=17), dict(init=2)]
    for kw in bad:
        a = dict(n_loc=4, S_w=32, systems=1, p=0.15, d=0.5, m=1, n_dec=2)
        a.update(kw)
        with pytest.raises(P.PcpdError) as e:
            P.PaperScheme(**a)
        assert e.value.code == P.PCPD_EINVAL
    with P.PaperScheme(4, 32, 1, 0.15, 0.5) as h:
        with pytest.raises(P.PcpdError):
            h.run(10, [5, 3])
        with pytest.raises(P.PcpdError):
            h.run(10, [11])
        with pytest.raises(P.PcpdError):
            h.run(1 << 32)
        h.run(10, [0, 10])
        with pytest.raises(P.PcpdError):
            h.run(5, [12, 12])
        h.run(5, [10, 15])          # the current step may be recorded again as the first entry
        assert h.num_records == 4 and h.step == 15
        c = h.counts()
        assert c[1] == c[2]


def test_paper_scheme_near_the_step_counter_limit(P, oracle_mod):
    """Steps just below 2^32: the stream block index n_w*t/4 passes 2^32 and its high bits go to
    the counter's tag word; the run must end exactly at 2^32 - 1 and be refused beyond."""
    n_loc, S_w, systems = 5, 64, 2
    step0 = (1 << 32) - 1 - 77
    rng = np.random.default_rng(8)
    st = (rng.random((systems, 32 * n_loc * S_w)) < 0.6).astype(np.uint8)
    with P.PaperScheme(n_loc, S_w, systems, 0.15, 0.5, 1, 2, seed=99) as h:
        h.set_lattice(sites_to_words(st, n_loc, S_w), step0)
        h.run(77, [step0, step0 + 40, step0 + 77])
        got = h.counts()
        lat = words_to_sites(h.lattice(), n_loc, S_w)
        with pytest.raises(P.PcpdError):
            h.run(1)
    ref = st.copy()
    want = oracle_mod.paper_run(ref, n_loc, S_w, 0.15, 0.5, 1, 2, 99, step0, step0 + 77,
                                [step0, step0 + 40, step0 + 77])
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(lat, ref)


@pytest.mark.parametrize("m,n_dec,p,S_w", [(1, 2, 0.15, 64), (2, 2, 0.2, 32), (3, 3, 0.1, 64), (5, 1, 0.3, 32)])
def test_paper_scheme_across_block_index_2_32(P, oracle_mod, m, n_dec, p, S_w):
    """A run across the step where the stream's block index B = n_w*t/4 reaches 2^32: the
    kernel forms most of a block's first three rounds once per thread for each value of
    B >> 32, and a group of four steps whose blocks straddle 2^32 takes the full counter.
    n_w = 5 and 6 straddle inside a group, n_w = 8 reaches 2^32 at a group start; m = 5 runs
    the kernel with (m, n_dec) read at run time."""
    n_loc, systems = 4, 3
    n_w = m + n_dec + 2
    t_cross = ((1 << 32) * 4 + n_w - 1) // n_w          # first step whose blocks have B >= 2^32
    step0 = t_cross - 37
    rng = np.random.default_rng(31 + m)
    st = (rng.random((systems, 32 * n_loc * S_w)) < 0.7).astype(np.uint8)
    d = 0.5
    recs = [step0 + 10, t_cross, step0 + 90]
    with P.PaperScheme(n_loc, S_w, systems, p, d, m, n_dec, seed=2024) as h:
        h.set_lattice(sites_to_words(st, n_loc, S_w), step0)
        h.run(90, recs)
        got = h.counts()
        lat = words_to_sites(h.lattice(), n_loc, S_w)
    ref = st.copy()
    want = oracle_mod.paper_run(ref, n_loc, S_w, p, d, m, n_dec, 2024, step0, step0 + 90, recs)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(lat, ref)


def test_paper_scheme_largest_system_that_fits_shared_memory(P, oracle_mod):
    """The longest ring one CTA can hold (n_loc*S_w words up to the shared-memory limit), one
    sampled system against the oracle; one more local word per thread is refused."""
    import torch
    optin = getattr(torch.cuda.get_device_properties(0), "shared_memory_per_block_optin", 232448)
    S_w = 64
    n_loc = optin // (4 * S_w)
    systems, steps = 3, 3 * n_loc
    with P.PaperScheme(n_loc, S_w, systems, 0.15, 0.5, 1, 2, seed=4) as h:
        h.run(steps, [steps])
        got = h.counts(per_system=True)[1]
        lat = h.lattice()
    for s in (0, 2):
        ref = np.ones((1, 32 * n_loc * S_w), np.uint8)
        want = oracle_mod.paper_run(ref, n_loc, S_w, 0.15, 0.5, 1, 2, 4, 0, steps, [steps], sys0=s)
        assert int(got[0, s]) == int(want[0])
        np.testing.assert_array_equal(words_to_sites(lat[s:s + 1], n_loc, S_w), ref)
    with pytest.raises(P.PcpdError):
        P.PaperScheme(n_loc + 1, S_w, 1, 0.15, 0.5)


def test_paper_scheme_records_at_launch_boundaries(P):
    """Runs longer than one launch (2^20 steps): a record exactly at a launch boundary is taken
    once, and the result does not depend on where the calls split the run."""
    n_loc, S_w, systems = 4, 32, 2
    edge = 1 << 20
    recs = [0, edge - 1, edge, edge + 1, edge + 100]
    with P.PaperScheme(n_loc, S_w, systems, 0.01, 1.0, 1, 0, seed=5) as a:   # d = 1: no absorption
        a.run(edge + 100, recs)
        ca, la = a.counts(per_system=True), a.lattice()
        assert a.num_records == len(recs)
    with P.PaperScheme(n_loc, S_w, systems, 0.01, 1.0, 1, 0, seed=5) as b:
        b.run(700001, [0])
        b.run(edge + 100 - 700001, recs[1:])
        cb, lb = b.counts(per_system=True), b.lattice()
    np.testing.assert_array_equal(ca[0], cb[0])
    np.testing.assert_array_equal(ca[1], cb[1])
    np.testing.assert_array_equal(la, lb)
    # d = 1 conserves particles in every system
    assert np.all(ca[1] == ca[1][0:1, :])
