"""Replicas across ranks (CPU, gloo, world size 2): disjoint seeds per rank, exact integer
sums of the occupation records, maximum of the timings.  The GPU path shards the same way
with no data-path collective."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_1301_6082_gb300.replicas import combine, replica_seed
    L, S, p, d = 90, 64, 0.15, 0.5
    seed = replica_seed(1, rank)
    rec = [O.substep_of_time(L, t) for t in (1, 5, 20)]
    st = O.init_state(L, S, O.MODE_FULL, seed)
    tot, _, _ = O.run(st, p, d, seed, 0, rec[-1], rec, threads=1)
    sums, maxes = combine(dist, [int(x) for x in tot], [0.5 + rank])
    if rank == 0:
        np.save(out_path, np.array(sums + [int(maxes[0] * 10)], dtype=np.int64))
    dist.destroy_process_group()


def test_replicas_sum_exactly_over_two_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / "sums.npy")
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    got = np.load(out)
    # independent recomputation of both replicas on this process
    from oracle import oracle as O
    from paper_1301_6082_gb300.replicas import replica_seed
    L, S, p, d = 90, 64, 0.15, 0.5
    rec = [O.substep_of_time(L, t) for t in (1, 5, 20)]
    want = np.zeros(3, dtype=np.int64)
    seeds = [replica_seed(1, r) for r in range(2)]
    assert seeds[0] != seeds[1]
    outs = []
    for s in seeds:
        st = O.init_state(L, S, O.MODE_FULL, s)
        tot, _, _ = O.run(st, p, d, s, 0, rec[-1], rec, threads=1)
        want += tot.astype(np.int64)
        outs.append(tot)
    assert not np.array_equal(outs[0], outs[1])     # the replicas are different systems
    np.testing.assert_array_equal(got[:3], want)
    assert got[3] == 15                              # max over ranks of 0.5 + rank


def test_single_process_combine_is_identity():
    from paper_1301_6082_gb300.replicas import combine, replica_seed
    assert combine(None, [3, 4], [1.5]) == ([3, 4], [1.5])
    assert replica_seed(1, 0) == 1 and replica_seed(1, 1) == 1 + 1_000_003
