"""CPU-side checks of the boundary: the library builds for sm_103a, loads, exports every
entry point include/pcpd.h declares, and its host-only helpers (thresholds, time) agree with
the oracle's.  No kernel is launched here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1301_6082_gb300 import build, pcpd
    build.build()
    return pcpd.load()


def declared_functions(header: str = "pcpd.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pcpd_\w+)\s*\(", src)))


def test_every_header_is_checked():
    assert sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")) == \
        ["pcpd.h", "pcpd_pipes.h"]


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_1301_6082_gb300 import pcpd
    bound = {n for n, _, _ in pcpd.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_pipe_rate_library_exports_its_header():
    from paper_1301_6082_gb300 import build, pipes
    build.build_pipes()
    plib = pipes.load()
    names = declared_functions("pcpd_pipes.h")
    assert names == ["pcpd_pipe_count", "pcpd_pipe_rate"]
    for n in names:
        assert hasattr(plib, n), n
    assert plib.pcpd_pipe_count() == len(pipes.OPS)


def test_thresholds_match_oracle(lib, oracle_mod):
    from paper_1301_6082_gb300 import pcpd
    rng = np.random.default_rng(3)
    cases = [(0.15, 0.5), (0.11, 0.1), (0.18, 0.9), (1.0, 0.0), (0.0, 1.0), (0.3, 0.0)]
    cases += [(float(a), float(b)) for a, b in rng.random((200, 2))]
    for p, d in cases:
        assert pcpd.thresholds(p, d) == oracle_mod.thresholds(p, d)[:2], (p, d)
    with pytest.raises(pcpd.PcpdError):
        pcpd.thresholds(-0.1, 0.5)


def test_substep_of_time_matches_oracle(lib, oracle_mod):
    from paper_1301_6082_gb300 import pcpd
    for L in (3, 4, 10, 1024, 65536, 1 << 22, 999999):
        for t in (0, 1, 2, 1000, 10**5, 10**6):
            assert pcpd.substep_of_time(L, t) == oracle_mod.substep_of_time(L, t)


def test_tuple_substep_of_time_matches_oracle(lib, oracle_mod):
    from paper_1301_6082_gb300 import pcpd
    for n in (3, 4):
        for L in (n + 1, 10, 1024, 65536, 999999):
            for t in (0, 1, 2, 1000, 10**6):
                assert pcpd.substep_of_time(L, t, n) == oracle_mod.substep_of_time(L, t, n)
    assert pcpd.substep_of_time(4, 10, 4) == 0          # shorter than one window
    assert pcpd.substep_of_time(100, 10, 5) == 0        # no such tuple size


def test_paper_thresholds_match_oracle(lib, oracle_mod):
    from paper_1301_6082_gb300 import pcpd
    rng = np.random.default_rng(11)
    for _ in range(300):
        m, n_dec = int(rng.integers(0, 17)), int(rng.integers(0, 17))
        d = int(rng.integers(0, (1 << m) + 1)) / float(1 << m)
        p = float(rng.random()) / float(1 << n_dec)
        assert pcpd.paper_thresholds(p, d, m, n_dec) == oracle_mod.paper_thresholds(p, d, m, n_dec), (p, d, m, n_dec)
    for bad in ((0.3, 0.5, 1, 2), (0.1, 0.3, 2, 0), (0.1, 0.5, 17, 0), (-0.1, 0.5, 1, 0)):
        with pytest.raises(pcpd.PcpdError):
            pcpd.paper_thresholds(*bad)
        with pytest.raises(ValueError):
            oracle_mod.paper_thresholds(*bad)


def test_thresholds_property_random_doubles(lib, oracle_mod):
    """Library and oracle agree on the thresholds for arbitrary doubles in [0, 1] (including
    the edges and values one ulp from them)."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    from paper_1301_6082_gb300 import pcpd

    @hyp.settings(max_examples=400, deadline=None)
    @hyp.given(st.floats(0.0, 1.0), st.floats(0.0, 1.0))
    def check(p, d):
        assert pcpd.thresholds(p, d) == oracle_mod.thresholds(p, d)[:2]
    check()


def test_no_cuda_device_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1301_6082_gb300 import pcpd
    with pytest.raises(pcpd.PcpdError) as e:
        pcpd.Pcpd(64, 64, 0.1, 0.5)
    assert e.value.code == pcpd.PCPD_ENODEV


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1301_6082_gb300")
    pat = re.compile(r"^\s*(from|import)\s+oracle\b|liboracle|pcpd_oracle", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                assert not pat.search(open(os.path.join(dirpath, f)).read()), f


def test_c_example_builds_and_fails_loudly_without_a_device():
    """The plain C example links against the library; on a machine without a CUDA device it
    reports the library's error instead of computing anything."""
    import subprocess
    import torch
    from paper_1301_6082_gb300 import build as B
    exe = B.build_example()
    if torch.cuda.is_available():
        return   # the GPU test covers the run itself
    r = subprocess.run([exe, "64", "32", "0.15", "0.5"], capture_output=True, text=True)
    assert r.returncode == 6 and "pcpd error 6" in r.stderr


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding passes across the ABI has the header's size and field offsets
    (a C program compiled against include/pcpd.h prints them)."""
    import subprocess
    from paper_1301_6082_gb300 import pcpd
    structs = {"pcpd_params": pcpd.Params, "pcpd_plan_info": pcpd.PlanInfo,
               "pcpd_server_config": pcpd.ServerConfig, "pcpd_server_stats": pcpd.ServerStats,
               "pcpd_paper_params": pcpd.PaperParams}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pcpd.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, key, val = line.split()
            got[(name, key)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_oracle_does_not_use_the_product():
    """The oracle shares no code with the CUDA path: it imports no package module and includes
    none of the library's headers or sources."""
    pat = re.compile(r"paper_1301_6082_gb300|pcpd\.h|pcpd_kernels|pcpd_engine|pcpd_capi|libpcpd")
    odir = os.path.join(ROOT, "oracle")
    for f in os.listdir(odir):
        if f.endswith((".py", ".c", ".h")):
            assert not pat.search(open(os.path.join(odir, f)).read()), f


class _FakeCudaTensor:
    """Stands in for a CUDA tensor: the allocation-free sweep's binding must refuse a buffer
    by its size before any device call."""
    is_cuda = True

    def __init__(self, words, contiguous=True):
        self.words, self.contig = words, contiguous

    def is_contiguous(self):
        return self.contig

    def numel(self):
        return self.words

    def element_size(self):
        return 4

    def data_ptr(self):
        raise AssertionError("the binding reached the device call")


def test_noalloc_binding_refuses_bad_buffers_before_any_launch():
    import torch
    from paper_1301_6082_gb300 import pcpd
    L, S = 1001, 64
    ok = _FakeCudaTensor((S // 32) * L)
    with pytest.raises(pcpd.PcpdError) as e:
        pcpd.sweep_noalloc(_FakeCudaTensor((S // 32) * L - 1), ok, L, S, 0.1, 0.5, 1, 0, 5)
    assert e.value.code == pcpd.PCPD_EINVAL and "lat_in" in str(e.value)
    with pytest.raises(pcpd.PcpdError) as e:
        pcpd.sweep_noalloc(ok, _FakeCudaTensor(10), L, S, 0.1, 0.5, 1, 0, 5)
    assert "lat_out" in str(e.value)
    with pytest.raises(pcpd.PcpdError) as e:
        pcpd.sweep_noalloc(_FakeCudaTensor((S // 32) * L, contiguous=False), ok, L, S, 0.1, 0.5, 1, 0, 5)
    assert "contiguous" in str(e.value)
    cpu = torch.zeros((S // 32) * L, dtype=torch.int32)
    with pytest.raises(pcpd.PcpdError) as e:
        pcpd.sweep_noalloc(cpu, ok, L, S, 0.1, 0.5, 1, 0, 5)
    assert "CUDA" in str(e.value)


def test_pair_density_entry_point_checks_its_arguments(lib):
    """pcpd_pair_density (Sec. 5.3's pair density, exported so the binding only marshals) is
    reachable through ctypes and refuses a missing handle or output before touching a device."""
    from paper_1301_6082_gb300 import pcpd
    out = (C.c_double * 4)()
    assert lib.pcpd_pair_density(None, out, 4) == pcpd.PCPD_EINVAL
    assert lib.pcpd_pair_density(None, None, 0) == pcpd.PCPD_EINVAL
    assert "NULL" in lib.pcpd_last_error().decode()
