"""The autotuner picks among tile plans by timing them; every plan gives the same bits, so
the tuned handle must reproduce the default plan's lattice exactly."""
import numpy as np
import pytest

from paper_1301_6082_gb300.workloads import INIT_HALF

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


@pytest.mark.parametrize("L,S", [(65536, 256), (5000, 128)])
def test_autotuned_plan_is_valid_and_bit_identical(P, L, S):
    best = P.autotune(L, S, 0.15, 0.5, trial_substeps=64)
    assert best["rate"] > 0 and best["plan_threads"] in (128, 256, 512)
    a = P.Pcpd(L, S, 0.15, 0.5, seed=5, init=INIT_HALF, plan_threads=best["plan_threads"],
               plan_seg_sites=best["plan_seg_sites"], plan_tau=best["plan_tau"])
    b = P.Pcpd(L, S, 0.15, 0.5, seed=5, init=INIT_HALF)
    c = P.Pcpd(L, S, 0.15, 0.5, seed=5, init=INIT_HALF, autotune=True)   # cached plan
    for s in (a, b, c):
        s.run(4, [2, 4])
    np.testing.assert_array_equal(a.lattice(), b.lattice())
    np.testing.assert_array_equal(c.lattice(), b.lattice())
    np.testing.assert_array_equal(a.counts(), b.counts())
