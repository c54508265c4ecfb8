"""Sharding one ensemble by group range (pcpd_params.group0) on the GPU: instances that hold
disjoint group ranges of the same seed reproduce the run of the whole ensemble bit for bit
(records sum exactly, lattices are the ensemble's rows), alone, in batches, and across two
processes that combine their records over gloo -- the multi-GPU path, run here as two
processes on one GPU whose kernels never wait on one another."""
import os
import socket

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


@pytest.mark.parametrize("L,S,p,d,init,tup,mcs", [
    (1000, 256, 0.15, 0.5, INIT_HALF, 2, 40),      # whole-ring tiles, 4 columns per tile
    (65536, 256, 0.11, 0.1, INIT_FULL, 2, 50),     # segmented tiles, several epochs
    (3001, 512, 0.2, 0.4, INIT_HALF, 3, 30),       # TCPD
])
def test_two_group_ranges_equal_the_whole_ensemble(P, oracle_mod, L, S, p, d, init, tup, mcs):
    seed = 99
    times = [1, mcs // 2, mcs]
    whole = P.Pcpd(L, S, p, d, seed=seed, init=init, tuple_n=tup, per_sample=True)
    whole.run(mcs, times)
    half = S // 2
    parts = [P.Pcpd(L, half, p, d, seed=seed, init=init, tuple_n=tup, group0=g0, per_sample=True)
             for g0 in (0, half // 32)]
    for h in parts:
        h.run(mcs, times)
    np.testing.assert_array_equal(parts[0].counts() + parts[1].counts(), whole.counts())
    np.testing.assert_array_equal(parts[0].pair_counts() + parts[1].pair_counts(), whole.pair_counts())
    lat = whole.lattice()
    G2 = half // 32
    np.testing.assert_array_equal(parts[0].lattice(), lat[:G2])
    np.testing.assert_array_equal(parts[1].lattice(), lat[G2:])
    for r in range(len(times)):
        ps = whole.sample_counts(r)
        np.testing.assert_array_equal(parts[1].sample_counts(r), ps[half:])
    # the upper shard against the oracle, from the initial state
    g0 = half // 32
    st = oracle_mod.init_state(L, 32, init, seed, g0)
    subs = [oracle_mod.substep_of_time(L, t, tup) for t in times]
    oracle_mod.run(st, p, d, seed, 0, subs[-1], subs, group0=g0, tuple_n=tup)
    np.testing.assert_array_equal(lat[g0], oracle_mod.pack(st)[0])
    for h in parts + [whole]:
        h.close()


def test_batch_members_with_group_offsets(P):
    L, S, p, d, seed, mcs = 5000, 256, 0.2, 0.3, 5, 25
    times = [5, mcs]
    whole = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF)
    whole.run(mcs, times)
    b = P.Batch()
    ids = [b.add(L, 128, p, d, seed, mcs, times, init=INIT_HALF, group0=g0) for g0 in (0, 4)]
    b.run()
    np.testing.assert_array_equal(b.counts(ids[0]) + b.counts(ids[1]), whole.counts())
    np.testing.assert_array_equal(np.concatenate([b.lattice(i) for i in ids]), whole.lattice())
    b.close()
    whole.close()


def test_group_offset_must_be_whole_phase_groups(P):
    with pytest.raises(P.PcpdError):
        P.Pcpd(100, 64, 0.1, 0.5, group0=2)
    with pytest.raises(P.PcpdError):
        P.Pcpd(100, 64, 0.1, 0.5, group0=(1 << 26) - 1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


SHARD = dict(L=20000, S=512, p=0.15, d=0.5, seed=3, mcs=30, times=[2, 10, 30])


def _rank(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_1301_6082_gb300 import pcpd
    from paper_1301_6082_gb300.replicas import combine, shard_groups
    c = SHARD
    g0, n = shard_groups(c["S"] // 32, world, rank)
    sim = pcpd.Pcpd(c["L"], 32 * n, c["p"], c["d"], seed=c["seed"], group0=g0)
    sim.run(c["mcs"], c["times"])
    sums, _ = combine(dist, [int(x) for x in sim.counts()] + [int(x) for x in sim.pair_counts()], [0.0])
    np.save(out_path + f".{rank}.npy", sim.lattice())
    sim.close()
    if rank == 0:
        np.save(out_path, np.array(sums, dtype=np.int64))
    dist.destroy_process_group()


def test_two_processes_sum_to_the_one_gpu_run(P, tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "sums.npy")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    got = np.load(out)
    c = SHARD
    whole = P.Pcpd(c["L"], c["S"], c["p"], c["d"], seed=c["seed"])
    whole.run(c["mcs"], c["times"])
    np.testing.assert_array_equal(got[:3], whole.counts().astype(np.int64))
    np.testing.assert_array_equal(got[3:], whole.pair_counts().astype(np.int64))
    lat = np.concatenate([np.load(out + f".{r}.npy") for r in range(2)])
    np.testing.assert_array_equal(lat, whole.lattice())
    whole.close()
