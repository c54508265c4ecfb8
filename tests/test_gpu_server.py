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


def test_cancel_queued_and_running_requests(P):
    """A queued request fails at once when cancelled; a running one at the end of its round,
    giving its memory back; the others' results are unaffected."""
    import time
    from paper_1301_6082_gb300.workloads import INIT_HALF
    sv = P.Server(hbm_budget_bytes=1 << 30, max_active=1, chunk_attempts=1 << 22)
    long_id = sv.submit(65536, 1024, 0.15, 0.5, 3, 100000, [100000])        # many rounds
    queued_id = sv.submit(2000, 64, 0.15, 0.5, 4, 50, [50])
    short_id = sv.submit(3000, 64, 0.2, 0.4, 5, 30, [10, 30], init=INIT_HALF, keep_lattice=True)
    sv.cancel(queued_id)
    assert sv.poll(queued_id) == 3
    for _ in range(200):                       # wait until the long request is on the GPU
        if sv.poll(long_id) == 1:
            break
        time.sleep(0.01)
    sv.cancel(long_id)
    sv.wait_idle()
    assert sv.poll(long_id) == 3
    with pytest.raises(P.PcpdError) as e:
        sv.result(long_id)
    assert "cancelled" in str(e.value)
    with pytest.raises(P.PcpdError):
        sv.cancel(short_id)                    # already finished
    c, lat, _, _ = sv.result(short_id)
    a = P.Pcpd(3000, 64, 0.2, 0.4, seed=5, init=INIT_HALF, jit=-1)
    a.run(30, [10, 30])
    np.testing.assert_array_equal(c, a.counts())
    np.testing.assert_array_equal(lat, a.lattice())
    st = sv.stats()
    assert st["failed"] == 2 and st["completed"] == 1 and st["mem_used_bytes"] == 0
    sv.stop()
