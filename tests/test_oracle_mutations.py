"""The pins must catch plausible mistakes.  Each case plants one mistake in a temporary
copy of the oracle's C source (on the CPU), rebuilds it, and checks that at least one of
the pin tests fails on the planted copy while all of them pass on the real oracle."""
import importlib.util
import os
import shutil
import subprocess

import pytest

import tests.test_oracle_exact as TE
import tests.test_oracle_invariants as TI
import tests.test_oracle_philox as TP
import tests.test_oracle_thresholds as TT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pcpd_oracle.c")

MUTANTS = {
    "philox_nine_rounds": ("round < 10", "round < 9"),
    "fission_target_is_partner": ("uint8_t *t = o ? sa : sc;", "uint8_t *t = o ? sc : sa;"),
    "annihilate_without_pair": ("} else if (*sb == 1 && *q == 1) {\n        if (u < t_da)",
                                "} else if (*sb == 1 || *q == 1) {\n        if (u < t_da)"),
    "rate_p_not_p_times_1_minus_d": ("double scaled_a = p * (1.0 - d);", "double scaled_a = p;"),
    "phase_always_zero": ("return (uint32_t)(((uint64_t)out[0] * (uint64_t)L) >> 32);", "return 0u;"),
    "windows_cover_wrap": ("const uint32_t L = jb->L, K = L / 3u;", "const uint32_t L = jb->L, K = (L + 2u) / 3u;"),
    "diffusion_swaps_a_c": ("*sb = *q;\n        *q = tmp;", "*sb = *sb;\n        *sa = *sc; *sc = tmp; (void)q;"),
    "time_floor_not_ceil": ("return (uint64_t)((num + K - 1) / K);", "return (uint64_t)(num / K);"),
    "pair_wrong_neighbour": ("pc += row[i] & row[(i + 1u) % jb->L];", "pc += row[i] & row[(i + 2u) % jb->L];"),
}


def _mutant_module(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    d = tmp_path / name
    d.mkdir()
    csrc = d / "pcpd_oracle.c"
    csrc.write_text(src.replace(old, new))
    so = d / "liboracle.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-pthread", str(csrc), "-o", str(so), "-lm"])
    spec = importlib.util.spec_from_file_location(f"oracle_mut_{name}", os.path.join(ROOT, "oracle", "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC = str(csrc)
    mod._LIB_PATH = str(so)
    return mod


def _pins(mod):
    """The pin checks, as (name, callable) pairs."""
    yield "philox_vs_triton", lambda: TP.test_philox_matches_triton_interpreter(mod)
    yield "thresholds_exact", lambda: TT.test_thresholds_vs_exact_rationals(mod, 0.15, 0.5)
    yield "threshold_specials", lambda: TT.test_threshold_special_values(mod)
    yield "substep_of_time", lambda: TT.test_substep_of_time(mod)
    yield "phase_law", lambda: TT.test_phase_is_uniform_law(mod)
    yield "bookkeeping", lambda: TI.test_particle_number_bookkeeping(mod, 0.15, 0.5)
    yield "d1_conserves", lambda: TI.test_d1_conserves_particles_per_sample(mod, 64)
    yield "p1_d0_closed_form", lambda: TI.test_p1_d0_first_substep_closed_form(mod)
    yield "binomial_first_substep", lambda: TI.test_full_lattice_first_substep_binomial(mod, 0.15, 0.5)
    for L in (4, 5, 8, 9):
        yield f"exact_chain_L{L}", (lambda L=L: TE.test_schedule_oracle_matches_exact_chain(mod, L, 0.15, 0.5))
    yield "pair_density_exact_L7", lambda: TE.test_pair_density_matches_exact_chain(mod, 7)


def _caught(mod):
    failed = []
    for name, fn in _pins(mod):
        try:
            fn()
        except (AssertionError, ValueError):
            failed.append(name)
    return failed


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    old, new = MUTANTS[name]
    mod = _mutant_module(tmp_path, name, old, new)
    failed = _caught(mod)
    assert failed, f"planted mistake {name} passed every pin"


def test_real_oracle_passes_every_pin(oracle_mod):
    assert _caught(oracle_mod) == []
