"""Serving with continuous batching: requests submitted while others run are admitted as
slots and memory free up, their work shares engine launches, and every result is
bit-identical to the same request run alone."""
import time

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


def test_results_same_alone_and_in_the_mix(P):
    rng = np.random.default_rng(8)
    reqs = []
    for i in range(24):
        L = int(round(2 ** rng.uniform(6, 14)))
        S = int(2 ** rng.integers(5, 9))
        p, d = float(rng.uniform(0.05, 0.25)), float(rng.uniform(0.1, 0.9))
        mcs = int(rng.integers(5, 60))
        rec = sorted(set([1, max(1, mcs // 2), mcs]))
        init = INIT_FULL if i % 2 else INIT_HALF
        reqs.append((L, S, p, d, 900 + i, mcs, rec, init))
    # a small memory budget and few slots force queueing; a small chunk forces many rounds,
    # so requests start, interleave and finish in different rounds
    budget = 6 * (2 * (1 << 14) * 8 * 4 + 8192)
    sv = P.Server(hbm_budget_bytes=budget, max_active=5, chunk_attempts=1 << 20)
    ids = []
    for j, (L, S, p, d, seed, mcs, rec, init) in enumerate(reqs):
        ids.append(sv.submit(L, S, p, d, seed, mcs, rec, init=init, keep_lattice=True))
        if j % 6 == 5:
            time.sleep(0.01)   # later requests arrive while earlier ones are on the GPU
    sv.wait_idle()
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["rounds"] > 3
    for rid, (L, S, p, d, seed, mcs, rec, init) in zip(ids, reqs):
        counts, lat, latency, queue = sv.result(rid)
        alone = P.Pcpd(L, S, p, d, seed=seed, init=init)
        alone.run(mcs, rec)
        np.testing.assert_array_equal(counts, alone.counts())
        np.testing.assert_array_equal(lat, alone.lattice())
        assert latency >= queue >= 0.0
        alone.close()
    sv.stop()


def test_server_rejects_bad_requests(P):
    sv = P.Server(max_active=2, chunk_attempts=1 << 20)
    with pytest.raises(P.PcpdError):
        sv.submit(100, 48, 0.1, 0.5, 1, 10)
    with pytest.raises(P.PcpdError):
        sv.submit(100, 32, 0.1, 0.5, 1, 10, [20])
    rid = sv.submit(100, 32, 0.1, 0.5, 1, 10, [10])
    c, _, _, _ = sv.result(rid)
    assert c.shape == (1,)
    sv.stop()
