"""Failure detection on the GPU without a GPU fault: a dependency flag that nothing sets
makes the engine's bounded wait give up; the kernel records a timeout code and returns, the
host reports PCPD_ETIMEOUT, and the context keeps working."""
import time

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


def test_dependency_wait_times_out_and_context_survives(P):
    t0 = time.perf_counter()
    rc = P.dev_timeout_test(200_000_000)     # ~0.1 s of GPU clock
    dt = time.perf_counter() - t0
    assert rc == P.PCPD_ETIMEOUT, P.load().pcpd_last_error()
    assert dt < 30.0
    # the context is still usable: a small run afterwards works and is reproducible
    a = P.Pcpd(200, 32, 0.15, 0.5, seed=3)
    a.run(5, [5])
    b = P.Pcpd(200, 32, 0.15, 0.5, seed=3)
    b.run(5, [5])
    np.testing.assert_array_equal(a.lattice(), b.lattice())


def test_allocation_failure_is_reported_and_the_context_survives(P):
    """A lattice larger than the device's free memory (2^29 sites x 2^14 samples, two buffers:
    2.2 TB) is refused before any allocation (PCPD_ENOMEM); the device keeps working."""
    with pytest.raises(P.PcpdError) as e:
        P.Pcpd(1 << 29, 1 << 14, 0.15, 0.5)
    assert e.value.code == P.PCPD_ENOMEM and "free" in str(e.value)
    with pytest.raises(P.PcpdError) as e:
        P.PaperScheme(32, 1024, 1 << 24, 0.15, 0.5)     # 2^24 systems of 128 KiB
    assert e.value.code == P.PCPD_ENOMEM
    sim = P.Pcpd(1000, 64, 0.15, 0.5)
    sim.run(5, [5])
    assert sim.counts()[0] > 0
    sim.close()


def test_injected_allocation_failure(P):
    """Host-side fault injection: with PCPD_INJECT_ALLOC_FAILURE=2 the second large allocation
    of the process fails (nothing is allocated), the call reports PCPD_ENOMEM and later calls
    work."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = (
        "import sys; sys.path.insert(0, sys.argv[1])\n"
        "from paper_1301_6082_gb300 import pcpd\n"
        "a = pcpd.Pcpd(1000, 64, 0.15, 0.5)\n"
        "try:\n"
        "    pcpd.Pcpd(1000, 64, 0.15, 0.5)\n"
        "    print('no failure')\n"
        "except pcpd.PcpdError as e:\n"
        "    print('code', e.code, 'injected' in str(e))\n"
        "c = pcpd.Pcpd(2000, 32, 0.2, 0.5)\n"
        "c.run(3, [3]); a.run(3, [3])\n"
        "print('ok', int(c.counts()[0]) > 0, int(a.counts()[0]) > 0)\n")
    env = dict(os.environ, PCPD_INJECT_ALLOC_FAILURE="2")
    r = subprocess.run([sys.executable, "-c", script, root], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.strip().splitlines()
    assert lines[-2] == "code 2 True" and lines[-1] == "ok True True", lines
