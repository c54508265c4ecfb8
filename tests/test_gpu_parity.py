"""GPU parity: the CUDA path through the C ABI against the CPU oracle, bit-exact (this is
integer bit work: lattices and occupation counts must be identical)."""
import numpy as np
import pytest

from paper_1301_6082_gb300.workloads import INIT_EMPTY, INIT_FULL, INIT_HALF, log_times

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1301_6082_gb300 import build, pcpd
    build.build()
    pcpd.load()
    return pcpd


def _oracle_run(O, L, S, p, d, seed, init, n_end, rec_sub, per_sample=False, group0=0, state=None, n_begin=0):
    st = O.init_state(L, S, init, seed, group0) if state is None else state
    tot, ps, _ = O.run(st, p, d, seed, n_begin, n_end, rec_sub, per_sample=per_sample, group0=group0)
    return st, tot, ps


def test_device_philox_matches_oracle(P, oracle_mod):
    import torch
    rng = np.random.default_rng(5)
    n = 100_003
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    dc = torch.from_numpy(ctr.view(np.int32)).cuda()
    out = torch.zeros_like(dc)
    for seed in (1, 0xDEADBEEFCAFEF00D):
        P.dev_philox(dc, seed, out, n)
        got = out.cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got, oracle_mod.philox(ctr, seed))


def _scalar_masks(words, td, tda):
    planes = words[:, 1:]   # P31..P0
    n = words.shape[0]
    lanes = np.arange(32, dtype=np.uint64)
    u = np.zeros((n, 32), dtype=np.uint64)
    for i in range(32):
        m = 31 - i
        u |= ((planes[:, i:i + 1].astype(np.uint64) >> lanes) & 1) << np.uint64(m)
    D = (u < td)
    A = (u >= td) & (u < tda)
    w = (1 << lanes).astype(np.uint64)
    return (D * w).sum(1).astype(np.uint32), (A * w).sum(1).astype(np.uint32)


@pytest.mark.parametrize("td,tda", [(0, 0), (0, 2**32), (2**32, 2**32), (2**31, 2**31 + 1),
                                    (1, 2), (2**32 - 1, 2**32), (0x19999999, 0x32F1A9FB),
                                    (0x80000000, 0x93333333), (0xE6666666, 0xEB020C49),
                                    (12345, 12345), (0x40000000, 0xC0000000)])
def test_rate_masks_exhaustive_vs_scalar(P, td, tda):
    # P10: the MSB-first plane compare equals the scalar u < T for every lane; words drawn
    # so that many lanes share long prefixes with the thresholds (the early-exit paths).
    import torch
    rng = np.random.default_rng(td ^ (tda >> 1))
    n = 20000
    words = rng.integers(0, 2**32, size=(n, 33), dtype=np.uint64).astype(np.uint32)
    for t in (td, tda):
        if t < 2**32:
            # make lanes of some items equal T on a random number of top bits
            idx = rng.choice(n, n // 2, replace=False)
            for it in idx[: n // 4]:
                k = rng.integers(1, 33)
                for i in range(k):
                    m = 31 - i
                    bit = (t >> m) & 1
                    lanes = rng.integers(0, 2**32, dtype=np.uint64)
                    words[it, 1 + i] = np.uint32((words[it, 1 + i] & ~np.uint32(lanes)) | (np.uint32(lanes) if bit else 0))
    dw = torch.from_numpy(words.view(np.int32)).cuda()
    dm = torch.zeros((n, 3), dtype=torch.int32, device="cuda")
    P.dev_rate_masks(dw, td, tda, dm, n)
    got = dm.cpu().numpy().view(np.uint32)
    D, A = _scalar_masks(words, td, tda)
    np.testing.assert_array_equal(got[:, 0], D)
    np.testing.assert_array_equal(got[:, 1], A)
    np.testing.assert_array_equal(got[:, 2], words[:, 0])


def test_L1024_S64_full_run_bit_exact(P, oracle_mod):
    # The L=1024, 64-sample, d=.5, p=.15, seed-1 decay run over 2000 MCS, 32 records.
    L, S, d, p, seed = 1024, 64, 0.5, 0.15, 1
    ts = log_times(2000, 32)
    sim = P.Pcpd(L, S, p, d, seed=seed, per_sample=True)
    sim.run(ts[-1], ts)
    got = sim.counts()
    lat = sim.lattice()
    ps_gpu = np.stack([sim.sample_counts(r) for r in range(len(ts))])
    subs = [oracle_mod.substep_of_time(L, t) for t in ts]
    st = oracle_mod.init_state(L, S, INIT_FULL, seed)
    tot, ps, _, prs = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs, per_sample=True, pairs=True)
    np.testing.assert_array_equal(got, tot)
    np.testing.assert_array_equal(ps_gpu, ps)
    np.testing.assert_array_equal(sim.pair_counts(), prs)
    np.testing.assert_array_equal(lat, oracle_mod.pack(st))
    golden = np.loadtxt(__file__.replace("test_gpu_parity.py", "golden/pcpd_L1024_S64.txt"), dtype=np.uint64)
    np.testing.assert_array_equal(got, golden[:, 2])
    assert np.allclose(sim.density(), tot / (L * S))
    assert sim.time_mcs == 2000 and sim.substep == subs[-1]


@pytest.mark.parametrize("L,S,p,d,init", [
    (3, 32, 0.2, 0.3, INIT_HALF), (4, 64, 0.5, 0.0, INIT_FULL), (5, 32, 0.0, 1.0, INIT_HALF),
    (7, 96, 1.0, 0.0, INIT_FULL), (10, 32, 0.15, 0.5, INIT_HALF), (31, 160, 0.3, 0.7, INIT_HALF),
    (100, 64, 0.11, 0.1, INIT_FULL), (1000, 32, 0.18, 0.9, INIT_HALF), (3001, 64, 0.25, 0.5, INIT_HALF),
    (64, 32, 0.15, 0.5, INIT_EMPTY)])
def test_ring_small_bit_exact(P, oracle_mod, L, S, p, d, init):
    seed = 1000 + L
    ts = [0, 1, 2, 5, 13, 40]
    sim = P.Pcpd(L, S, p, d, seed=seed, init=init, per_sample=True)
    sim.run(ts[-1], ts)
    subs = [oracle_mod.substep_of_time(L, t) for t in ts]
    st, tot, ps = _oracle_run(oracle_mod, L, S, p, d, seed, init, subs[-1], subs, per_sample=True)
    np.testing.assert_array_equal(sim.counts(), tot)
    np.testing.assert_array_equal(np.stack([sim.sample_counts(r) for r in range(len(ts))]), ps)
    np.testing.assert_array_equal(sim.lattice(), oracle_mod.pack(st))


@pytest.mark.parametrize("L,seg,tau,threads", [(3000, 1000, 16, 256), (4099, 1500, 37, 128), (20000, 6001, 64, 512)])
def test_segmented_plan_bit_exact_and_plan_invariant(P, oracle_mod, L, seg, tau, threads):
    # Tiles with halos (temporal blocking) and a ragged last tile give the same bits as the
    # oracle and as the whole-ring plan.
    S, p, d, seed = 64, 0.15, 0.5, 77
    ts = [3, 17, 60]
    a = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF, plan_seg_sites=seg, plan_tau=tau, plan_threads=threads)
    a.run(ts[-1], ts)
    b = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF)
    b.run(ts[-1], ts)
    np.testing.assert_array_equal(a.lattice(), b.lattice())
    np.testing.assert_array_equal(a.counts(), b.counts())
    subs = [oracle_mod.substep_of_time(L, t) for t in ts]
    st = oracle_mod.init_state(L, S, INIT_HALF, seed)
    tot, _, _, prs = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs, pairs=True)
    np.testing.assert_array_equal(a.counts(), tot)
    np.testing.assert_array_equal(a.pair_counts(), prs)
    np.testing.assert_array_equal(b.pair_counts(), prs)
    np.testing.assert_array_equal(a.lattice(), oracle_mod.pack(st))


def test_default_plans_two_ctas_per_sm_alone_and_in_batches(P, oracle_mod):
    """A lone instance whose columns exceed one CTA's shared memory runs two 256-thread CTAs
    per SM (tau = 64), and so does the same instance in a batch (every batch member's tile fits
    half an SM). Both give the oracle's bits, and so does the one-CTA plan forced on a lone
    instance (one 512-thread CTA per SM, the largest tile, tau = 128)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    L, S, p, d, seed, mcs = 65536, 64, 0.15, 0.5, 5, 3
    times = [1, 2, 3]
    a = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF)
    pa = a.plan()
    assert pa["ring"] == 0 and pa["threads"] == 256 and pa["tau"] == 64 and pa["grid"] == 2 * sms, pa
    a.run(mcs, times)
    c = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF, plan_threads=512, plan_seg_sites=32768, plan_tau=128)
    pc = c.plan()
    assert pc["threads"] == 512 and pc["grid"] == sms, pc
    c.run(mcs, times)
    b = P.Batch()
    i = b.add(L, S, p, d, seed, mcs, times, init=INIT_HALF)
    b.run()
    subs = [oracle_mod.substep_of_time(L, t) for t in times]
    st = oracle_mod.init_state(L, S, INIT_HALF, seed)
    tot, _, _ = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs)
    for got in (a.counts(), c.counts(), b.counts(i)):
        np.testing.assert_array_equal(got, tot)
    np.testing.assert_array_equal(a.lattice(), oracle_mod.pack(st))
    np.testing.assert_array_equal(c.lattice(), oracle_mod.pack(st))
    a.close(), c.close(), b.close()


@pytest.mark.parametrize("L,S,tuple_n", [(20000, 64, 2), (12001, 96, 2), (30011, 32, 3)])
def test_short_columns_cut_into_segments_when_sms_would_idle(P, oracle_mod, L, S, tuple_n):
    """Columns that fit one CTA but are fewer than the SMs: a lone instance cuts them into
    segments (ragged last one included) instead of whole-column tiles; same bits as the
    oracle, with records inside and at the end of the run."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    p, d, seed = 0.2, 0.4, 21
    a = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF, tuple_n=tuple_n)
    plan = a.plan()
    assert S // 32 < sms and plan["ring"] == 0 and plan["n_seg"] >= 2 and plan["core"] >= 4096, plan
    times = [2, 5, 9]
    a.run(times[-1], times)
    subs = [oracle_mod.substep_of_time(L, t, tuple_n) for t in times]
    st = oracle_mod.init_state(L, S, INIT_HALF, seed)
    tot, _, _, prs = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs, pairs=True, tuple_n=tuple_n)
    np.testing.assert_array_equal(a.counts(), tot)
    np.testing.assert_array_equal(a.pair_counts(), prs)
    np.testing.assert_array_equal(a.lattice(), oracle_mod.pack(st))
    a.close()


def test_resume_from_saved_state_is_exact(P):
    L, S, p, d, seed = 777, 96, 0.2, 0.4, 3
    a = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF)
    a.run(30)
    b = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF)
    b.run(12)
    saved, n = b.lattice(), b.substep
    c = P.Pcpd(L, S, p, d, seed=seed, init=INIT_EMPTY)
    c.set_lattice(saved, n)
    assert c.time_mcs == 12
    c.run(18)
    np.testing.assert_array_equal(a.lattice(), c.lattice())


def test_bad_arguments_raise(P):
    with pytest.raises(P.PcpdError):
        P.Pcpd(2, 32, 0.1, 0.1)
    with pytest.raises(P.PcpdError):
        P.Pcpd(100, 48, 0.1, 0.1)
    with pytest.raises(P.PcpdError):
        P.Pcpd(100, 32, 1.5, 0.1)
    sim = P.Pcpd(100, 32, 0.1, 0.1)
    with pytest.raises(P.PcpdError):
        sim.run(10, [5, 5])
    with pytest.raises(P.PcpdError):
        sim.run(10, [11])
    sim.run(10, [10])
    with pytest.raises(P.PcpdError):
        sim.run(5, [3])


def _sampled_groups_check(P, O, L, S, p, d, seed, n1, groups, plan=None):
    """Run the GPU for n1 sub-steps at full size, then check the chosen groups against the
    oracle started from the initial state; then splice: oracle from the GPU state at n1 for
    a few more sub-steps vs the GPU."""
    sim = P.Pcpd(L, S, p, d, seed=seed, **(plan or {}))
    sim.run_substeps(n1)
    lat1 = sim.lattice()
    for g in groups:
        st = O.init_state(L, 32, INIT_FULL, seed, g)
        O.run(st, p, d, seed, 0, n1, group0=g)
        np.testing.assert_array_equal(lat1[g], O.pack(st)[0], err_msg=f"group {g} after {n1} sub-steps")
    dn = 3
    sim.run_substeps(dn)
    lat2 = sim.lattice()
    for g in groups:
        st = O.unpack(lat1[g:g + 1])
        O.run(st, p, d, seed, n1, n1 + dn, group0=g)
        np.testing.assert_array_equal(lat2[g], O.pack(st)[0], err_msg=f"splice group {g}")


@pytest.mark.parametrize("d,p", [(0.1, 0.11), (0.5, 0.15), (0.9, 0.18)])
def test_L65536_S4096_sampled_groups(P, oracle_mod, d, p):
    _sampled_groups_check(P, oracle_mod, 65536, 4096, p, d, 1, 4, [0, 5, 127])


def test_L4194304_S1024_sampled_groups(P, oracle_mod):
    _sampled_groups_check(P, oracle_mod, 1 << 22, 1024, 0.15, 0.5, 1, 2, [0, 31])


def test_live_handles_with_different_tiles(P):
    # handles with different tile sizes alive at once (the kernel's shared-memory limit is
    # process-wide state): create all, then run all, each equal to a lone run
    spec = [(50000, 32, 0.2, 0.5), (1000, 64, 0.1, 0.3), (20000, 32, 0.15, 0.9), (300, 32, 0.3, 0.1)]
    sims = [P.Pcpd(L, S, p, d, seed=7 + i, init=INIT_HALF) for i, (L, S, p, d) in enumerate(spec)]
    for s in sims:
        s.run(3, [3])
    for i, ((L, S, p, d), s) in enumerate(zip(spec, sims)):
        a = P.Pcpd(L, S, p, d, seed=7 + i, init=INIT_HALF)
        a.run(3, [3])
        np.testing.assert_array_equal(s.lattice(), a.lattice())
        a.close()
        s.close()


@pytest.mark.parametrize("L,seg,d,p", [(3000, 1000, 0.5, 0.15), (3000, 1000, 0.1, 0.11), (1000, 0, 0.9, 0.18),
                                       (20000, 6000, 0.3, 0.7), (777, 0, 0.25, 0.05)])
def test_runtime_specialised_sweep_bit_exact(P, oracle_mod, L, seg, d, p):
    # the sweep compiled at run time for this (T_D, T_DA) pair == the generic sweep == oracle
    S, seed = 64, 31
    ts = [2, 9, 25]
    a = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF, plan_seg_sites=seg, plan_tau=32 if seg else 0, jit=1)
    assert a.plan()["jit"] == 1
    a.run(ts[-1], ts)
    b = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF, plan_seg_sites=seg, plan_tau=32 if seg else 0, jit=-1)
    assert b.plan()["jit"] == 0
    b.run(ts[-1], ts)
    np.testing.assert_array_equal(a.lattice(), b.lattice())
    np.testing.assert_array_equal(a.counts(), b.counts())
    subs = [oracle_mod.substep_of_time(L, t) for t in ts]
    st = oracle_mod.init_state(L, S, INIT_HALF, seed)
    tot, _, _, prs = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs, pairs=True)
    np.testing.assert_array_equal(a.counts(), tot)
    np.testing.assert_array_equal(a.pair_counts(), prs)
    np.testing.assert_array_equal(a.lattice(), oracle_mod.pack(st))


@pytest.mark.parametrize("jit", [-1, 1])
def test_many_groups_multi_column_tiles(P, oracle_mod, jit):
    # 2048 groups on a short ring: tiles hold 4 whole columns each (one phase group); sampled
    # groups against the oracle, per-sample records against the oracle for those groups
    L, S, p, d, seed = 100, 65536, 0.2, 0.4, 9
    ts = [3, 10]
    sim = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF, per_sample=True, jit=jit)
    assert sim.plan()["gpi"] == 4
    sim.run(ts[-1], ts)
    lat = sim.lattice()
    ps = np.stack([sim.sample_counts(r) for r in range(len(ts))])
    subs = [oracle_mod.substep_of_time(L, t) for t in ts]
    for g in (0, 1, 2, 3, 4, 777, 2047):
        st = oracle_mod.init_state(L, 32, INIT_HALF, seed, g)
        _, pso, _ = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs, per_sample=True, group0=g)
        np.testing.assert_array_equal(lat[g], oracle_mod.pack(st)[0], err_msg=f"group {g}")
        np.testing.assert_array_equal(ps[:, 32 * g:32 * g + 32], pso, err_msg=f"group {g}")
    tot = sim.counts()
    np.testing.assert_array_equal(tot, ps.sum(1))


def test_record_now_after_resume(P, oracle_mod):
    L, S, p, d, seed = 500, 64, 0.15, 0.5, 21
    a = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF)
    a.run(7)
    saved, n = a.lattice(), a.substep
    b = P.Pcpd(L, S, p, d, seed=seed, init=INIT_EMPTY)
    b.set_lattice(saved, n)
    b.run(5, [7, 9, 12])        # 7 = the current time: records the restored state
    c = b.counts()
    st = oracle_mod.init_state(L, S, INIT_HALF, seed)
    subs = [oracle_mod.substep_of_time(L, t) for t in (7, 9, 12)]
    tot, _, _ = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs)
    np.testing.assert_array_equal(c, tot)
    assert b.num_records == 3 and list(b.record_times()) == [7, 9, 12]


def test_late_splice_deep_into_a_run(P, oracle_mod):
    # 2^21 + 12345 sub-steps of the L=65536 lattice (1024 samples) on the specialised sweep,
    # then three more sub-steps checked against the oracle started from the GPU state
    L, S, p, d, seed = 65536, 1024, 0.15, 0.5, 1
    n1 = (1 << 21) + 12345
    sim = P.Pcpd(L, S, p, d, seed=seed, jit=1)
    assert sim.plan()["jit"] == 1
    sim.run_substeps(n1)
    lat1 = sim.lattice()
    sim.run_substeps(3)
    lat2 = sim.lattice()
    for g in (0, 13, 31):
        st = oracle_mod.unpack(lat1[g:g + 1])
        oracle_mod.run(st, p, d, seed, n1, n1 + 3, group0=g)
        np.testing.assert_array_equal(lat2[g], oracle_mod.pack(st)[0], err_msg=f"group {g}")


def test_substep_counter_near_its_limit(P, oracle_mod):
    # the sub-step index is a 32-bit Philox counter word: a run may reach 2^32 - 1 and no further
    L, S, p, d, seed = 600, 64, 0.2, 0.3, 5
    n0 = (1 << 32) - 60
    st0 = oracle_mod.init_state(L, S, INIT_HALF, seed)
    sim = P.Pcpd(L, S, p, d, seed=seed)
    sim.set_lattice(oracle_mod.pack(st0), n0)
    sim.run_substeps(59)
    st = st0.copy()
    oracle_mod.run(st, p, d, seed, n0, n0 + 59)
    np.testing.assert_array_equal(sim.lattice(), oracle_mod.pack(st))
    with pytest.raises(P.PcpdError):
        sim.run_substeps(2)


def test_plans_exist_for_every_lattice_size_near_the_shared_memory_limit(P):
    """Every L from ring-sized through a few segments gets a plan that fits (the 16-byte
    rounding of segment cores must not push a tile past the budget), and runs."""
    for L in list(range(30011, 80000, 997)) + [39328, 39329, 39330, 78655, 78660]:
        with P.Pcpd(L, 32, 0.15, 0.5, seed=2, jit=-1) as sim:
            sim.run_substeps(3)
            sim.sync()
            plan = sim.plan()
            assert plan["ring"] == 1 or plan["core"] + 2 * plan["halo"] <= 60000


def test_maximum_samples_sampled_groups(P, oracle_mod):
    """2^22 samples (the largest accepted) on a short ring: 131072 groups, whole-ring tiles."""
    L, S, p, d, seed, n1 = 64, 1 << 22, 0.15, 0.5, 5, 10
    sim = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF)
    sim.run_substeps(n1)
    lat = sim.lattice()
    for g in (0, 4097, (S // 32) - 1):
        st = oracle_mod.init_state(L, 32, INIT_HALF, seed, g)
        oracle_mod.run(st, p, d, seed, 0, n1, group0=g)
        np.testing.assert_array_equal(lat[g], oracle_mod.pack(st)[0], err_msg=f"group {g}")
    sim.close()


def _popcount_total(words: np.ndarray) -> int:
    if hasattr(np, "bitwise_count"):
        return int(np.bitwise_count(words).sum(dtype=np.uint64))
    lut = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint8)
    b = words.view(np.uint8).reshape(-1)
    return int(sum(int(lut[b[i:i + (1 << 26)]].sum(dtype=np.uint64)) for i in range(0, b.size, 1 << 26)))


def test_maximum_lattice_length_closed_forms(P):
    """L = 2^30 - 1 (the longest accepted ring), checked by properties that hold at any size:
    p = 1, d = 0 from full empties every window's pair in the first sub-step (N = L - 2K per
    sample, exactly), and d = 1 conserves the particle number."""
    L, S = (1 << 30) - 1, 32
    K = L // 3
    sim = P.Pcpd(L, S, 1.0, 0.0, seed=3, jit=-1)
    sim.run_substeps(1)
    n1 = _popcount_total(sim.lattice())
    assert n1 == S * (L - 2 * K)
    sim.close()
    sim = P.Pcpd(L, S, 0.3, 1.0, seed=4, init=INIT_HALF, jit=-1)
    n0 = _popcount_total(sim.lattice())
    sim.run_substeps(2)
    assert _popcount_total(sim.lattice()) == n0
    sim.close()


def test_async_lattice_copies_match_waiting_ones(P):
    import torch
    L, S = 5000, 64
    a = P.Pcpd(L, S, 0.2, 0.4, seed=12, init=INIT_HALF)
    a.run(7)
    start, n = a.lattice(), a.substep
    a.run(9)
    want = a.lattice()
    pinned = torch.empty((S // 32, L), dtype=torch.int32, pin_memory=True)
    buf = pinned.numpy().view(np.uint32)
    buf[...] = start
    b = P.Pcpd(L, S, 0.2, 0.4, seed=12, init=INIT_EMPTY, stream=torch.cuda.Stream())
    b.set_lattice(buf, n, wait=False)
    b.run(9)
    b.lattice(out=buf, wait=False)
    b.sync()
    np.testing.assert_array_equal(buf, want)


def test_c_example_program_matches_the_binding(P):
    """The plain C user of the C ABI (examples/pcpd_decay.c) prints the same densities as the
    Python binding for the same run (PCPD and TCPD)."""
    import subprocess
    from paper_1301_6082_gb300 import build as B
    exe = B.build_example()
    for tup in (2, 3):
        r = subprocess.run([exe, "3000", "64", "0.15", "0.5", str(tup), "200", "9"], capture_output=True,
                           text=True, check=True)
        rows = np.array([[float(x) for x in line.split()] for line in r.stdout.strip().splitlines()])
        t = rows[:, 0].astype(np.uint64)
        sim = P.Pcpd(3000, 64, 0.15, 0.5, seed=9, tuple_n=tup)
        sim.run(200, t)
        np.testing.assert_allclose(rows[:, 1], sim.density(), rtol=0, atol=1e-9)
        np.testing.assert_allclose(rows[:, 2], sim.pair_density(), rtol=0, atol=1e-9)
        sim.close()


def test_tile_count_limit_is_enforced(P):
    # a work item carries its tile index in 24 bits: plans beyond 2^24 - 1 tiles are refused
    with pytest.raises(P.PcpdError) as e:
        P.Pcpd(1 << 22, 1 << 22, 0.1, 0.1, plan_seg_sites=1024, plan_tau=16)
    assert e.value.code == P.PCPD_EINVAL and "tiles" in str(e.value)


def test_no_tile_is_shorter_than_its_halo(P, oracle_mod):
    """A tile's halo may reach only into its two neighbours, whose epoch flags it waits on; a
    ragged last tile shorter than the halo (L = 3001 in tiles of 1000: a 1-site last tile)
    would let a halo reach two tiles away and race with a tile it does not wait for.  The
    planner evens such tiles out (4 tiles of at most 752 sites) and refuses tiles that cannot
    hold a halo; the evened plan runs several epochs bit-exact to the oracle."""
    L, S, p, d, seed = 3001, 64, 0.15, 0.5, 31
    a = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF, plan_seg_sites=1000, plan_tau=20, jit=-1)
    plan = a.plan()
    assert plan["ring"] == 0 and plan["n_seg"] == 4 and plan["core"] == 752, plan
    assert L - 3 * plan["core"] >= plan["halo"]
    ts = [5, 30, 60]
    a.run(ts[-1], ts)
    subs = [oracle_mod.substep_of_time(L, t) for t in ts]
    st = oracle_mod.init_state(L, S, INIT_HALF, seed)
    tot, _, _ = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs)
    np.testing.assert_array_equal(a.counts(), tot)
    np.testing.assert_array_equal(a.lattice(), oracle_mod.pack(st))
    a.close()
    with pytest.raises(P.PcpdError) as e:
        P.Pcpd(3000, 64, p, d, plan_seg_sites=40, plan_tau=20, jit=-1)
    assert e.value.code == P.PCPD_EINVAL and "halo" in str(e.value)
