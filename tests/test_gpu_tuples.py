"""GPU parity of the n-tuple processes (TCPD n = 3, QCPD n = 4; windows of n+1 sites) against
the oracle, bit for bit: counts, per-sample counts, pair counts and lattices, on whole-ring and
segmented plans, the generic and the runtime-specialised sweep, batches and the server."""
import numpy as np
import pytest

from paper_1301_6082_gb300.workloads import INIT_EMPTY, INIT_FULL, INIT_HALF

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


def _oracle(O, L, S, p, d, seed, init, ts, n, per_sample=False):
    subs = [O.substep_of_time(L, t, n) for t in ts]
    st = O.init_state(L, S, init, seed)
    tot, ps, _, prs = O.run(st, p, d, seed, 0, subs[-1], subs, per_sample=per_sample, pairs=True, tuple_n=n)
    return st, tot, ps, prs, subs


@pytest.mark.parametrize("n", [3, 4])
def test_L1024_S64_full_run_bit_exact(P, oracle_mod, n):
    L, S, d, p, seed = 1024, 64, 0.5, 0.15, 1
    ts = [0, 1, 2, 4, 8, 16, 32, 64, 128, 300]
    for jit in (-1, 1):
        sim = P.Pcpd(L, S, p, d, seed=seed, per_sample=True, tuple_n=n, jit=jit)
        assert sim.plan()["jit"] == (1 if jit == 1 else 0)
        sim.run(ts[-1], ts)
        st, tot, ps, prs, subs = _oracle(oracle_mod, L, S, p, d, seed, INIT_FULL, ts, n, per_sample=True)
        np.testing.assert_array_equal(sim.counts(), tot)
        np.testing.assert_array_equal(np.stack([sim.sample_counts(r) for r in range(len(ts))]), ps)
        np.testing.assert_array_equal(sim.pair_counts(), prs)
        np.testing.assert_array_equal(sim.lattice(), oracle_mod.pack(st))
        assert sim.substep == subs[-1] and sim.time_mcs == ts[-1]
        assert P.substep_of_time(L, ts[-1], n) == subs[-1]
        sim.close()


@pytest.mark.parametrize("n,L,S,p,d,init", [
    (3, 4, 32, 0.2, 0.3, INIT_HALF), (3, 5, 64, 1.0, 0.0, INIT_FULL), (3, 11, 32, 0.0, 1.0, INIT_HALF),
    (3, 97, 96, 0.15, 0.5, INIT_HALF), (3, 2999, 64, 0.3, 0.7, INIT_HALF), (3, 64, 32, 0.15, 0.5, INIT_EMPTY),
    (4, 5, 32, 0.2, 0.3, INIT_HALF), (4, 6, 64, 1.0, 0.0, INIT_FULL), (4, 13, 32, 0.05, 0.1, INIT_HALF),
    (4, 101, 160, 0.25, 0.5, INIT_HALF), (4, 3001, 64, 0.11, 0.9, INIT_HALF)])
def test_ring_small_bit_exact(P, oracle_mod, n, L, S, p, d, init):
    seed = 500 + L + n
    ts = [0, 1, 2, 5, 13, 40]
    sim = P.Pcpd(L, S, p, d, seed=seed, init=init, per_sample=True, tuple_n=n)
    sim.run(ts[-1], ts)
    st, tot, ps, prs, _ = _oracle(oracle_mod, L, S, p, d, seed, init, ts, n, per_sample=True)
    np.testing.assert_array_equal(sim.counts(), tot)
    np.testing.assert_array_equal(np.stack([sim.sample_counts(r) for r in range(len(ts))]), ps)
    np.testing.assert_array_equal(sim.pair_counts(), prs)
    np.testing.assert_array_equal(sim.lattice(), oracle_mod.pack(st))


@pytest.mark.parametrize("n,L,seg,tau,threads,jit", [
    (3, 3000, 1000, 16, 256, -1), (3, 4099, 1500, 37, 128, 1), (4, 3001, 1000, 20, 256, -1),
    (4, 20000, 6001, 64, 512, 1), (3, 20000, 6000, 64, 512, -1)])
def test_segmented_plan_bit_exact_and_plan_invariant(P, oracle_mod, n, L, seg, tau, threads, jit):
    S, p, d, seed = 64, 0.15, 0.5, 77
    ts = [3, 17, 60]
    a = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF, plan_seg_sites=seg, plan_tau=tau, plan_threads=threads,
               tuple_n=n, jit=jit)
    plan = a.plan()
    assert plan["ring"] == 0 and plan["halo"] == n * tau + n + 2
    a.run(ts[-1], ts)
    b = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF, tuple_n=n, jit=-1)
    b.run(ts[-1], ts)
    np.testing.assert_array_equal(a.lattice(), b.lattice())
    st, tot, _, prs, _ = _oracle(oracle_mod, L, S, p, d, seed, INIT_HALF, ts, n)
    np.testing.assert_array_equal(a.counts(), tot)
    np.testing.assert_array_equal(a.pair_counts(), prs)
    np.testing.assert_array_equal(b.counts(), tot)
    np.testing.assert_array_equal(a.lattice(), oracle_mod.pack(st))


@pytest.mark.parametrize("n", [3, 4])
def test_L65536_S4096_sampled_groups_and_splice(P, oracle_mod, n):
    """The bench-sized lattice: groups checked from the start and after a splice."""
    L, S, p, d, seed, n1 = 65536, 4096, 0.15, 0.5, 1, 4
    sim = P.Pcpd(L, S, p, d, seed=seed, tuple_n=n)
    sim.run_substeps(n1)
    lat1 = sim.lattice()
    groups = [0, 33, 127]
    for g in groups:
        st = oracle_mod.init_state(L, 32, INIT_FULL, seed, g)
        oracle_mod.run(st, p, d, seed, 0, n1, group0=g, tuple_n=n)
        np.testing.assert_array_equal(lat1[g], oracle_mod.pack(st)[0], err_msg=f"group {g}")
    sim.run_substeps(3)
    lat2 = sim.lattice()
    for g in groups:
        st = oracle_mod.unpack(lat1[g:g + 1])
        oracle_mod.run(st, p, d, seed, n1, n1 + 3, group0=g, tuple_n=n)
        np.testing.assert_array_equal(lat2[g], oracle_mod.pack(st)[0], err_msg=f"splice group {g}")


def test_resume_is_exact(P):
    for n in (3, 4):
        a = P.Pcpd(777, 96, 0.2, 0.4, seed=3, init=INIT_HALF, tuple_n=n)
        a.run(30)
        b = P.Pcpd(777, 96, 0.2, 0.4, seed=3, init=INIT_HALF, tuple_n=n)
        b.run(12)
        c = P.Pcpd(777, 96, 0.2, 0.4, seed=3, init=INIT_EMPTY, tuple_n=n)
        c.set_lattice(b.lattice(), b.substep)
        assert c.time_mcs == 12
        c.run(18)
        np.testing.assert_array_equal(a.lattice(), c.lattice())


def test_batch_mixing_tuple_sizes_equals_lone_runs(P):
    spec = [(2000, 64, 0.15, 0.5, 2), (3001, 32, 0.2, 0.3, 3), (999, 96, 0.1, 0.7, 4), (40000, 32, 0.15, 0.5, 3),
            (5000, 64, 0.25, 0.1, 4), (700, 32, 0.3, 0.9, 2)]
    b = P.Batch()
    for i, (L, S, p, d, n) in enumerate(spec):
        b.add(L, S, p, d, 40 + i, 30, [5, 30], init=INIT_HALF, tuple_n=n)
    b.run()
    for i, (L, S, p, d, n) in enumerate(spec):
        a = P.Pcpd(L, S, p, d, seed=40 + i, init=INIT_HALF, tuple_n=n, jit=-1)
        a.run(30, [5, 30])
        np.testing.assert_array_equal(b.counts(i), a.counts())
        np.testing.assert_array_equal(b.pair_counts(i), a.pair_counts())
        np.testing.assert_array_equal(b.lattice(i), a.lattice())
        a.close()
    b.close()
    # a batch of one tuple size runs the engine specialised for it; same bits
    b2 = P.Batch()
    b2.add(3001, 32, 0.2, 0.3, 41, 30, [5, 30], init=INIT_HALF, tuple_n=3)
    b2.add(40000, 32, 0.15, 0.5, 43, 30, [5, 30], init=INIT_HALF, tuple_n=3)
    b2.run()
    a = P.Pcpd(40000, 32, 0.15, 0.5, seed=43, init=INIT_HALF, tuple_n=3, jit=-1)
    a.run(30, [5, 30])
    np.testing.assert_array_equal(b2.lattice(1), a.lattice())
    b2.close()


def test_server_request_with_tuples_equals_lone_run(P):
    sv = P.Server(hbm_budget_bytes=1 << 30, max_active=8, chunk_attempts=1 << 24)
    ids = [sv.submit(3000, 64, 0.15, 0.5, 9, 40, [10, 40], init=INIT_HALF, keep_lattice=True, tuple_n=n)
           for n in (2, 3, 4)]
    for rid, n in zip(ids, (2, 3, 4)):
        c, lat, _, _ = sv.result(rid)
        a = P.Pcpd(3000, 64, 0.15, 0.5, seed=9, init=INIT_HALF, tuple_n=n, jit=-1)
        a.run(40, [10, 40])
        np.testing.assert_array_equal(c, a.counts())
        np.testing.assert_array_equal(lat, a.lattice())
        a.close()
    sv.stop()


def test_bad_tuple_arguments(P):
    for kw in (dict(tuple_n=1), dict(tuple_n=5)):
        with pytest.raises(P.PcpdError):
            P.Pcpd(100, 32, 0.1, 0.1, **kw)
    with pytest.raises(P.PcpdError):
        P.Pcpd(4, 32, 0.1, 0.1, tuple_n=4)      # shorter than one window
    assert P.substep_of_time(4, 10, 4) == 0


@pytest.mark.parametrize("n,jit", [(3, -1), (4, 1)])
def test_many_groups_multi_column_tiles(P, oracle_mod, n, jit):
    # 2048 groups on a short ring: tiles hold 4 whole columns each; sampled groups and their
    # per-sample records against the oracle
    L, S, p, d, seed = 101, 65536, 0.2, 0.4, 19
    ts = [3, 10]
    sim = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF, per_sample=True, jit=jit, tuple_n=n)
    assert sim.plan()["gpi"] == 4
    sim.run(ts[-1], ts)
    lat = sim.lattice()
    ps = np.stack([sim.sample_counts(r) for r in range(len(ts))])
    subs = [oracle_mod.substep_of_time(L, t, n) for t in ts]
    for g in (0, 3, 5, 1030, 2047):
        st = oracle_mod.init_state(L, 32, INIT_HALF, seed, g)
        _, pso, _ = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs, per_sample=True, group0=g, tuple_n=n)
        np.testing.assert_array_equal(lat[g], oracle_mod.pack(st)[0], err_msg=f"group {g}")
        np.testing.assert_array_equal(ps[:, 32 * g:32 * g + 32], pso, err_msg=f"group {g}")
