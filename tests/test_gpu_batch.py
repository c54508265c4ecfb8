"""Batched heterogeneous instances in one persistent launch: every instance's records and
final lattice are bit-identical to the same instance run alone, and to the oracle."""
import numpy as np
import pytest

from paper_1301_6082_gb300.workloads import INIT_FULL, INIT_HALF, batch_instances

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


MIX = [  # L, S, p, d, seed, mcs, init, plan_seg_sites, plan_tau
    (1024, 64, 0.15, 0.5, 11, 40, INIT_FULL, 0, 0),
    (777, 96, 0.2, 0.3, 12, 25, INIT_HALF, 0, 0),
    (3000, 64, 0.11, 0.1, 13, 30, INIT_HALF, 1000, 16),     # segmented, ragged last tile
    (5, 32, 0.3, 0.7, 14, 50, INIT_FULL, 0, 0),
    (20000, 128, 0.18, 0.9, 15, 12, INIT_FULL, 6000, 32),   # segmented
    (65536, 64, 0.25, 0.5, 16, 3, INIT_HALF, 0, 0),         # segmented by the planner
    (4099, 32, 0.05, 0.0, 17, 20, INIT_HALF, 0, 0),
    (1024, 256, 1.0, 0.0, 18, 5, INIT_FULL, 0, 0),
]


def test_batch_equals_alone_and_oracle(P, oracle_mod):
    b = P.Batch()
    recs = []
    for (L, S, p, d, seed, mcs, init, seg, tau) in MIX:
        r = sorted(set([1, max(1, mcs // 3), mcs]))
        recs.append(r)
        b.add(L, S, p, d, seed, mcs, r, init=init, plan_seg_sites=seg, plan_tau=tau)
    b.run()
    for i, (L, S, p, d, seed, mcs, init, seg, tau) in enumerate(MIX):
        alone = P.Pcpd(L, S, p, d, seed=seed, init=init)
        alone.run(mcs, recs[i])
        np.testing.assert_array_equal(b.counts(i), alone.counts(), err_msg=f"instance {i}")
        np.testing.assert_array_equal(b.pair_counts(i), alone.pair_counts(), err_msg=f"pairs, instance {i}")
        lat = b.lattice(i)
        np.testing.assert_array_equal(lat, alone.lattice(), err_msg=f"instance {i}")
        alone.close()
        if L * S * mcs <= 3_000_000:
            subs = [oracle_mod.substep_of_time(L, t) for t in recs[i]]
            st = oracle_mod.init_state(L, S, init, seed)
            tot, _, _, prs = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs, pairs=True)
            np.testing.assert_array_equal(b.counts(i), tot, err_msg=f"oracle, instance {i}")
            np.testing.assert_array_equal(b.pair_counts(i), prs, err_msg=f"oracle pairs, instance {i}")
            np.testing.assert_array_equal(lat, oracle_mod.pack(st), err_msg=f"oracle, instance {i}")
    b.close()


def test_batch_more_than_one_launch(P):
    # 130 instances > 128 descriptors per launch: the batch runs as consecutive launches
    rng = np.random.default_rng(3)
    b = P.Batch()
    spec = []
    for i in range(130):
        L = int(rng.integers(30, 400))
        d, p = float(rng.choice([0.1, 0.5, 0.9])), float(rng.uniform(0.05, 0.25))
        spec.append((L, d, p))
        b.add(L, 32, p, d, 500 + i, 10, [5, 10], init=INIT_HALF)
    b.run()
    for i in (0, 77, 127, 128, 129):
        L, d, p = spec[i]
        a = P.Pcpd(L, 32, p, d, seed=500 + i, init=INIT_HALF)
        a.run(10, [5, 10])
        np.testing.assert_array_equal(b.counts(i), a.counts())
        np.testing.assert_array_equal(b.lattice(i), a.lattice())
        a.close()
    b.close()


def test_batch_workload_mix_sample(P):
    # a slice of the 512-instance mix (L log-uniform 2^10..2^18, 64/256/1024 samples), with
    # the step counts divided by 1000 to keep the test short; checked against lone runs
    mix = batch_instances(512, seed=1)[:24]
    b = P.Batch()
    for m in mix:
        b.add(m["L"], m["S"], m["p"], m["d"], m["seed"], max(1, m["mcs"] // 1000), [max(1, m["mcs"] // 1000)],
              init=m["init"])
    b.run()
    for i in (0, 5, 11, 23):
        m = mix[i]
        a = P.Pcpd(m["L"], m["S"], m["p"], m["d"], seed=m["seed"], init=m["init"])
        t = max(1, m["mcs"] // 1000)
        a.run(t, [t])
        np.testing.assert_array_equal(b.counts(i), a.counts())
        np.testing.assert_array_equal(b.lattice(i), a.lattice())
        a.close()
    b.close()


def test_batch_errors(P):
    b = P.Batch()
    with pytest.raises(P.PcpdError):
        b.add(100, 32, 0.1, 0.5, 1, 10, [11])
    with pytest.raises(P.PcpdError):
        b.add(100, 32, 0.1, 0.5, 1, 10, [5, 5])
    b.add(100, 32, 0.1, 0.5, 1, 10, [10])
    b.run()
    with pytest.raises(P.PcpdError):
        b.run()
    b.close()


def test_members_sharing_thresholds_run_a_specialised_kernel(P, oracle_mod):
    """Members that share (T_D, T_DA) and window width (the seeds of one p in a sweep) run in
    launches of the engine compiled for their pair; the rest on the generic kernel.  Same bits
    either way, and the same as the oracle."""
    spec = [  # L, S, p, d, seed, mcs, init, tuple
        (3000, 64, 0.15, 0.5, 21, 30, INIT_HALF, 2),
        (65536, 64, 0.15, 0.5, 22, 4, INIT_FULL, 2),   # segmented, same pair as the first
        (1000, 96, 0.15, 0.5, 23, 40, INIT_HALF, 2),
        (2000, 64, 0.2, 0.3, 24, 25, INIT_HALF, 2),     # a pair of its own
        (3001, 32, 0.15, 0.5, 25, 30, INIT_HALF, 3),    # same pair, other window width
        (3001, 32, 0.15, 0.5, 26, 30, INIT_FULL, 3),
    ]
    lattices = {}
    for mode in (1, -1):
        b = P.Batch()
        b.set_jit(mode)
        ids = []
        for L, S, p, d, seed, mcs, init, tup in spec:
            ids.append(b.add(L, S, p, d, seed, mcs, [mcs // 2, mcs], init=init, tuple_n=tup))
        b.run()
        if mode > 0:
            assert b.jit_launches == 2, b.jit_launches    # the PCPD pair and the TCPD pair
        else:
            assert b.jit_launches == 0
        lattices[mode] = [(b.counts(i), b.lattice(i)) for i in ids]
        b.close()
    for (c1, l1), (c2, l2) in zip(lattices[1], lattices[-1]):
        np.testing.assert_array_equal(c1, c2)
        np.testing.assert_array_equal(l1, l2)
    for (L, S, p, d, seed, mcs, init, tup), (c, lat) in zip(spec, lattices[1]):
        subs = [oracle_mod.substep_of_time(L, t, tup) for t in (mcs // 2, mcs)]
        st = oracle_mod.init_state(L, S, init, seed)
        tot, _, _ = oracle_mod.run(st, p, d, seed, 0, subs[-1], subs, tuple_n=tup)
        np.testing.assert_array_equal(c, tot)
        np.testing.assert_array_equal(lat, oracle_mod.pack(st))
