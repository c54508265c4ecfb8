"""The allocation-free sweep (pcpd_sweep_noalloc) against the allocating path.

Callers such as an application whose device memory all belongs to its own pool, or a
latency-critical loop that cannot afford cudaMalloc/cudaFree (they can synchronize the device
and fail on a fragmented heap), use this entry point; its scratch is a fixed array inside the
library.  The results must be bit-identical to pcpd_run_substeps on two calls in a row (the
second call reuses the scratch the first one left behind).  This file is collected last."""
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


@pytest.mark.parametrize("L,S,p,d,n1,n2", [
    # this entry point keeps the caller's unpadded layout (column pitch = L): with L % 4 != 0
    # and several columns, later columns start off a 16-byte boundary and take the plain-load
    # path instead of the bulk copy
    (1001, 64, 0.15, 0.5, 37, 90),          # whole-ring tiles, 2 columns, 1001 = 4*250 + 1
    (65538, 96, 0.2, 0.3, 70, 200),         # segmented tiles, 3 columns, 65538 = 4*16384 + 2
    (65536, 256, 0.11, 0.1, 130, 260),      # segmented tiles across several epochs
])
def test_noalloc_matches_allocating_path_twice(P, L, S, p, d, n1, n2):
    import torch
    seed = 4242
    ref = P.Pcpd(L, S, p, d, seed=seed, init=INIT_HALF)
    start = ref.lattice()
    ref.run_substeps(n1)
    want1 = ref.lattice()
    ref.run_substeps(n2)
    want2 = ref.lattice()
    ref.close()

    dev = torch.device("cuda")
    a = torch.from_numpy(start.view(np.int32).copy()).to(dev)
    b = torch.empty_like(a)
    P.sweep_noalloc(a, b, L, S, p, d, seed, 0, n1)          # first call
    got1 = b.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got1, want1)
    c = torch.empty_like(a)
    P.sweep_noalloc(b, c, L, S, p, d, seed, n1, n2)         # second call, continues the run
    got2 = c.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got2, want2)


def test_noalloc_rejects_oversized_work(P):
    import ctypes as C
    import torch
    a = torch.zeros(8, dtype=torch.int32, device="cuda")
    b = torch.zeros(8, dtype=torch.int32, device="cuda")
    # 2^22 samples on 65536 sites: 131072 columns x 2 segments, beyond the fixed scratch.  The
    # C entry point refuses before touching the (deliberately small) buffers; the binding
    # would refuse them earlier for their size, so the entry point is called directly.
    rc = P.load().pcpd_sweep_noalloc(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), 65536, 1 << 22,
                                     0.1, 0.5, 1, 0, 10, None)
    assert rc == P.PCPD_EINVAL and "scratch" in P.load().pcpd_last_error().decode()
    with pytest.raises(P.PcpdError) as e:   # and the binding refuses the small buffers themselves
        P.sweep_noalloc(a, b, 65536, 1 << 22, 0.1, 0.5, 1, 0, 10)
    assert e.value.code == P.PCPD_EINVAL and "lat_in" in str(e.value)
