"""GPU parity across tile epochs, at the plans the benchmark runs.

A lattice longer than one CTA's shared memory is cut into segment tiles that each run tau
sub-steps per residency (an epoch); a tile of epoch e starts only after its two neighbours
have published epoch e-1 through acquire/release flags.  These tests run the default plans
of the benchmark's workloads for several epochs in ONE launch sequence (no re-creation of
the handle in between), with every CTA of the persistent grid resident, and compare sampled
32-sample groups with the oracle started from the initial state (Eq. (1), Alg. 1 on the
window schedule).  The oracle is never restarted from GPU state here, so an error in an
early epoch cannot hide."""
import concurrent.futures as cf

import numpy as np
import pytest

from paper_1301_6082_gb300.workloads import INIT_FULL, INIT_HALF

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


def _oracle_groups(O, L, p, d, seed, n_end, groups, rec_sub=(), init=INIT_FULL, tuple_n=2):
    """Each sampled group advanced by the oracle from the initial state, one host thread per
    group (the oracle's C core runs outside the interpreter lock).  Returns, per group, the
    packed column and the per-sample record counts [R][32]."""
    def one(g):
        st = O.init_state(L, 32, init, seed, g)
        _, ps, _ = O.run(st, p, d, seed, 0, n_end, rec_sub, per_sample=True, threads=1, group0=g,
                         tuple_n=tuple_n)
        return O.pack(st)[0], ps
    with cf.ThreadPoolExecutor(max_workers=len(groups)) as ex:
        return list(ex.map(one, groups))


@pytest.mark.parametrize("d,p", [(0.1, 0.11), (0.5, 0.15), (0.9, 0.18)])
def test_L65536_S4096_bench_plan_several_epochs(P, oracle_mod, d, p):
    """The L = 65536, 4096-sample workload on its default plan (runtime-specialised sweep,
    two 256-thread CTAs per SM, tau = 64, three tiles per column) for 67 MCS = 202 sub-steps
    (epochs 0-3) in one run call, with per-sample records inside every epoch."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    L, S, seed = 65536, 4096, 1
    times = [1, 21, 43, 60, 67]
    sim = P.Pcpd(L, S, p, d, seed=seed, per_sample=True)
    plan = sim.plan()
    assert (plan["ring"], plan["threads"], plan["tau"], plan["n_seg"], plan["grid"], plan["jit"]) == \
        (0, 256, 64, 3, 2 * sms, 1), plan
    sim.run(times[-1], times)
    subs = [oracle_mod.substep_of_time(L, t) for t in times]
    assert subs[-1] > 3 * plan["tau"]
    lat = sim.lattice()
    ps = np.stack([sim.sample_counts(r) for r in range(len(times))])
    groups = [0, 63, 127]
    for g, (col, ps_o) in zip(groups, _oracle_groups(oracle_mod, L, p, d, seed, subs[-1], groups, subs)):
        np.testing.assert_array_equal(lat[g], col, err_msg=f"group {g} after {subs[-1]} sub-steps")
        np.testing.assert_array_equal(ps[:, 32 * g:32 * g + 32], ps_o, err_msg=f"records of group {g}")
    np.testing.assert_array_equal(sim.counts(), ps.sum(1, dtype=np.uint64))
    sim.close()


def test_L4194304_S1024_streamed_plan_several_epochs(P, oracle_mod):
    """The HBM-streamed L = 2^22, 1024-sample workload on its default plan for three epochs
    and a ragged fourth (2*tau + 5 sub-steps) in one call; groups 0 and 31 against the oracle
    from the full start."""
    L, S, p, d, seed = 1 << 22, 1024, 0.15, 0.5, 1
    sim = P.Pcpd(L, S, p, d, seed=seed)
    plan = sim.plan()
    assert plan["ring"] == 0 and plan["jit"] == 1 and plan["n_seg"] > 2, plan
    n1 = 2 * plan["tau"] + 5
    sim.run_substeps(n1)
    lat = sim.lattice()
    groups = [0, 31]
    for g, (col, _) in zip(groups, _oracle_groups(oracle_mod, L, p, d, seed, n1, groups)):
        np.testing.assert_array_equal(lat[g], col, err_msg=f"group {g} after {n1} sub-steps")
    sim.close()


def test_batch_members_segmented_several_epochs(P, oracle_mod):
    """Batch members on their batched plan (one 512-thread CTA per SM, tau = 128): a
    segmented PCPD lattice and a segmented TCPD lattice for more than two epochs each, beside
    whole-ring members, in one batch; every member against the oracle (records, per-sample
    records via the totals, final lattice)."""
    spec = [  # L, S, p, d, seed, mcs, init, tuple
        (65536, 64, 0.15, 0.5, 11, 90, INIT_FULL, 2),
        (60001, 32, 0.2, 0.3, 12, 70, INIT_HALF, 3),
        (3001, 64, 0.11, 0.1, 13, 200, INIT_HALF, 2),
        (777, 96, 0.18, 0.9, 14, 300, INIT_FULL, 4),
    ]
    b = P.Batch()
    idx = []
    for L, S, p, d, seed, mcs, init, tup in spec:
        times = sorted({1, mcs // 3, mcs // 2, mcs})
        idx.append((b.add(L, S, p, d, seed, mcs, times, init=init, tuple_n=tup), times))
    b.run()
    for (L, S, p, d, seed, mcs, init, tup), (i, times) in zip(spec, idx):
        subs = [oracle_mod.substep_of_time(L, t, tup) for t in times]
        if L > 50000:
            assert subs[-1] > 2 * 128 + 2, subs
        st = oracle_mod.init_state(L, S, init, seed)
        tot, _, _, prs = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs, pairs=True, tuple_n=tup)
        np.testing.assert_array_equal(b.counts(i), tot, err_msg=f"member {i}")
        np.testing.assert_array_equal(b.pair_counts(i), prs, err_msg=f"member {i}")
        np.testing.assert_array_equal(b.lattice(i), oracle_mod.pack(st), err_msg=f"member {i}")
    b.close()
