"""Sharding one ensemble by group range across ranks (CPU, gloo, world size 2): each rank
advances its own groups [group0, group0 + n) with the oracle, the ranks combine their
occupation records by an exact integer sum, and the sum equals the one-rank run of the
whole ensemble bit for bit.  The GPU path shards the same way (pcpd_params.group0) with no
data-path collective."""
import os
import socket

import numpy as np
import pytest

L, S, P_, D_, SEED = 90, 256, 0.15, 0.5, 7   # 8 groups = 2 phase groups


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path, init):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_1301_6082_gb300.replicas import combine, shard_groups
    g0, n = shard_groups(S // 32, world, rank)
    rec = [O.substep_of_time(L, t) for t in (1, 5, 20)]
    st = O.init_state(L, 32 * n, init, SEED, g0)
    tot, _, _, prs = O.run(st, P_, D_, SEED, 0, rec[-1], rec, threads=1, group0=g0, pairs=True)
    sums, maxes = combine(dist, [int(x) for x in tot] + [int(x) for x in prs], [0.5 + rank])
    np.save(out_path + f".{rank}.npy", O.pack(st))
    if rank == 0:
        np.save(out_path, np.array(sums + [int(maxes[0] * 10)], dtype=np.int64))
    dist.destroy_process_group()


@pytest.mark.parametrize("init", [0, 2])
def test_group_shards_sum_to_the_one_rank_run(tmp_path, init):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / "sums.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out, init), nprocs=2, start_method="spawn", join=True)
    got = np.load(out)
    from oracle import oracle as O
    rec = [O.substep_of_time(L, t) for t in (1, 5, 20)]
    st = O.init_state(L, S, init, SEED)
    tot, _, _, prs = O.run(st, P_, D_, SEED, 0, rec[-1], rec, threads=1, pairs=True)
    np.testing.assert_array_equal(got[:3], tot.astype(np.int64))
    np.testing.assert_array_equal(got[3:6], prs.astype(np.int64))
    assert got[6] == 15                              # max over ranks of 0.5 + rank
    lat = np.concatenate([np.load(out + f".{r}.npy") for r in range(2)])
    np.testing.assert_array_equal(lat, O.pack(st))   # the shards are the ensemble's groups


def test_shard_arithmetic():
    from paper_1301_6082_gb300.replicas import combine, shard_groups, weak_shard
    assert combine(None, [3, 4], [1.5]) == ([3, 4], [1.5])
    for total in (1, 3, 4, 8, 13, 128, 130):
        for world in (1, 2, 3, 4, 8):
            parts = [shard_groups(total, world, r) for r in range(world)]
            covered = [g for g0, n in parts for g in range(g0, g0 + n)]
            assert covered == list(range(total)), (total, world, parts)
            assert all(g0 % 4 == 0 for g0, n in parts if n)
    assert weak_shard(128, 3) == (384, 128)
    with pytest.raises(ValueError):
        weak_shard(6, 0)
