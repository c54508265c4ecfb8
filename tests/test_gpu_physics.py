"""Qualitative physics of the simulated process (no exact reference exists at these sizes).
The paper finds p_c < 1/4 for d = 1/4, 1/2, 3/4 (Sec. 4.3): at p = 1/4 the density must decay
faster than at criticality (effective decay exponent well above the critical value near 0.2,
on its way to the 1/2 of diffusion-limited pair annihilation), while deep in the active phase
it settles at a finite value."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("d", [0.25, 0.5, 0.75])
def test_subcritical_at_quarter_and_active_at_small_p(P, d):
    from paper_1301_6082_gb300.sweep import p_sweep
    out = p_sweep(d, (0.01, 0.25), 4096, 256, 20000, n_rec=12, seeds=(1,))
    sub, act = out[0.25], out[0.01]
    assert sub["rho"][-1] < 0.02 and np.all(np.diff(sub["rho"]) < 0), sub["rho"]
    assert sub["delta_eff"][1][-1] > 0.25, sub["delta_eff"]      # decays faster than critical
    assert act["rho"][-1] > 0.05, act["rho"]                      # a steady active density
    assert abs(act["delta_eff"][1][-1]) < 0.05, act["delta_eff"]
    assert np.all(sub["rho_pair"] <= sub["rho"]) and np.all(act["rho_pair"] <= act["rho"])
