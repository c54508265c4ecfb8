"""The index-checked debug build (libpcpd_debug.so, -DPCPD_DEBUG): on a spread of plans -- whole
rings, segmented tiles, multi-column tiles, the n-tuple windows, batches, the paper's scheme --
no kernel forms an out-of-range shared- or global-memory index, and the results equal the
release build's bit for bit (a stand-in for a memory sanitizer)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1301_6082_gb300 import pcpd
from paper_1301_6082_gb300.workloads import INIT_HALF
out = {"debug": pcpd.debug_build(), "runs": {}}
def h(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:16]
cases = [("ring", dict(L=1000, samples=64, p=0.15, d=0.5), 2),
         ("ring_odd", dict(L=3001, samples=96, p=0.3, d=0.7), 2),
         ("segments", dict(L=20000, samples=64, p=0.15, d=0.5, plan_seg_sites=6001, plan_tau=64), 2),
         ("multicol", dict(L=100, samples=65536, p=0.2, d=0.4), 2),
         ("tcpd_seg", dict(L=20000, samples=64, p=0.05, d=0.5, plan_seg_sites=6000, plan_tau=32), 3),
         ("qcpd_ring", dict(L=4099, samples=64, p=0.05, d=0.5), 4),
         ("L65536", dict(L=65536, samples=256, p=0.15, d=0.5), 2)]
for name, kw, n in cases:
    sim = pcpd.Pcpd(seed=7, init=INIT_HALF, jit=-1, tuple_n=n, **kw)
    sim.run(12, [3, 12])
    out["runs"][name] = [h(sim.lattice()), sim.counts().tolist(), sim.pair_counts().tolist(), pcpd.debug_check()]
    sim.close()
b = pcpd.Batch()
for i, (L, S, n) in enumerate([(2000, 64, 2), (3001, 32, 3), (40000, 32, 2), (999, 96, 4)]):
    b.add(L, S, 0.15, 0.5, 40 + i, 10, [10], init=INIT_HALF, tuple_n=n)
b.run()
out["runs"]["batch"] = [[h(b.lattice(i)) for i in range(4)], [b.counts(i).tolist() for i in range(4)], pcpd.debug_check()]
b.close()
for S_w, n_loc, spc in ((64, 32, 0), (32, 64, 0), (512, 4, 0), (64, 8, 3)):
    ps = pcpd.PaperScheme(n_loc, S_w, 5, 0.15, 0.5, seed=3, plan_spc=spc)
    ps.run(20 * n_loc, [n_loc, 20 * n_loc])
    out["runs"]["paper_%d_%d_%d" % (S_w, n_loc, spc)] = [h(ps.lattice()), ps.counts().tolist(), pcpd.debug_check()]
    ps.close()
print(json.dumps(out))
"""


def _run(lib):
    env = dict(os.environ, PCPD_LIB=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, env=env,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_finds_no_out_of_range_index_and_matches_release():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    from paper_1301_6082_gb300 import build
    rel = _run(build.build())
    dbg = _run(build.build(debug=True))
    assert dbg["debug"] and not rel["debug"]
    for name, res in dbg["runs"].items():
        assert res[-1] == 0, (name, res[-1])            # no failed index check
        assert res[:-1] == rel["runs"][name][:-1], name  # same bits as the release build
