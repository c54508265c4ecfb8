"""The seeded input generators: record times, the batch mix and the request stream have the
stated ranges, are deterministic per seed and (for the stream) Poisson at the stated rate."""
import math

import numpy as np

from paper_1301_6082_gb300.workloads import batch_instances, log_times, request_stream


def test_log_times_strictly_increasing_with_the_stated_ends():
    for t_max, n in ((2000, 32), (10**6, 100), (10, 30), (1, 1)):
        t = log_times(t_max, n)
        assert len(t) == n
        assert all(b > a for a, b in zip(t, t[1:]))
        if n > 1:
            assert t[0] == 1
            assert t[-1] == max(t_max, n)   # bumped past t_max only when n exceeds it
    t = log_times(10**6, 100)
    ratios = np.diff(np.log(t[40:]))   # past the small times where ceil rounding dominates
    assert np.allclose(ratios, math.log(10**6) / 99, rtol=0.05)


def test_batch_mix_ranges_and_determinism():
    mix = batch_instances(512, seed=1)
    assert mix == batch_instances(512, seed=1)
    assert mix != batch_instances(512, seed=2)
    L = np.array([m["L"] for m in mix])
    assert L.min() >= 2**10 and L.max() <= 2**18
    assert {m["S"] for m in mix} <= {64, 256, 1024}
    assert {m["d"] for m in mix} <= {0.1, 0.3, 0.5, 0.7, 0.9}
    assert all(0.05 <= m["p"] <= 0.25 for m in mix)
    assert all(10**3 <= m["mcs"] <= 10**5 for m in mix)
    assert [m["seed"] for m in mix] == list(range(1000, 1512))
    # log-uniform L: log2 L roughly uniform on [10, 18]
    assert abs(np.log2(L).mean() - 14.0) < 0.4


def test_request_stream_is_poisson_at_the_rate():
    reqs = request_stream(rate_hz=200.0, duration_s=60.0, seed=1)
    n = len(reqs)
    assert abs(n - 12000) < 5 * math.sqrt(12000)
    arr = np.array([r["arrival"] for r in reqs])
    assert np.all(np.diff(arr) > 0) and arr[-1] < 60.0
    gaps = np.diff(arr)
    assert abs(gaps.mean() - 1 / 200.0) < 5 * (1 / 200.0) / math.sqrt(len(gaps))
    assert all(2**10 <= r["L"] <= 2**20 and r["S"] in (64, 128, 256, 512, 1024, 2048, 4096) for r in reqs)
    scaled = request_stream(rate_hz=200.0, duration_s=1.0, seed=1, mcs_scale=1 / 600)
    assert all(r["mcs"] >= 1 for r in scaled)
