"""The algorithmic work per (window, group) item that the bench's roofline divides by: the
expected planes and Philox blocks under the per-item MSB-first early exit, against a direct
simulation of random 32-lane items (no GPU)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def planes_needed(u, T):
    """Planes (MSB first) after which u < T is decided, per lane: the first plane where u and T
    differ, or the point past which T has only zero bits (an equal prefix then means u >= T)."""
    x = (u ^ np.uint32(T)).astype(np.uint64)
    lz = np.full(x.shape, 32, dtype=np.int64)
    nz = x != 0
    lz[nz] = 31 - np.floor(np.log2(x[nz].astype(np.float64))).astype(np.int64)
    tz = (T & -T).bit_length() - 1
    return np.minimum(lz + 1, 32 - tz)


@pytest.mark.parametrize("d,p", [(0.1, 0.11), (0.5, 0.15), (0.9, 0.18), (0.3, 0.25)])
def test_expected_planes_and_blocks_match_simulation(oracle_mod, d, p):
    import bench
    td, tda, _ = oracle_mod.thresholds(p, d)
    _, blocks, planes, mul, logic = bench.algorithmic_ops_per_item(td, tda)
    rng = np.random.default_rng(7)
    n = 40000
    u = rng.integers(0, 1 << 32, size=(n, 32), dtype=np.uint64).astype(np.uint32)
    need = np.maximum(planes_needed(u, td), planes_needed(u, tda)).max(axis=1)   # per item
    # block 0 holds planes 31..29, block b >= 1 planes 32-4b .. 29-4b
    sim_blocks = 1 + sum((need > k).astype(np.int64) for k in (3, 7, 11, 15, 19, 23, 27, 31))
    sim_planes = need.astype(np.float64)
    se_b = sim_blocks.std() / np.sqrt(n)
    se_p = sim_planes.std() / np.sqrt(n)
    assert abs(sim_blocks.mean() - blocks) < 5 * se_b + 1e-9, (sim_blocks.mean(), blocks)
    assert abs(sim_planes.mean() - planes) < 5 * se_p + 1e-9, (sim_planes.mean(), planes)
    assert mul == pytest.approx(20.0 * blocks)
    assert logic == pytest.approx(20.0 * blocks + 2.0 * planes + 11.0)


def test_planes_needed_small_cases():
    u = np.array([0x80000000, 0x7FFFFFFF, 0x40000000, 0x00000000], dtype=np.uint32)
    # T = 2^31: decided after the first plane for every u
    assert planes_needed(u, 1 << 31).tolist() == [1, 1, 1, 1]
    # T = 0x40000001: 0x7FFFFFFF first differs at plane 3 (bit 29), 0x40000000 agrees on 31
    # planes and differs at the last, 0 differs at plane 2 (bit 30)
    assert planes_needed(u, 0x40000001).tolist() == [1, 3, 32, 2]
    # T = 0x40000000 (low 30 bits zero): an equal 2-bit prefix already means u >= T
    assert planes_needed(u, 0x40000000).tolist() == [1, 2, 2, 2]
