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
import tests.test_oracle_paper_scheme as TPS
import tests.test_oracle_tuples as TU

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pcpd_oracle.c")

MUTANTS = {
    "philox_nine_rounds": ("round < 10", "round < 9"),
    "fission_target_is_partner": ("const uint32_t target = o ? 0u : n;", "const uint32_t target = o ? n : 0u;"),
    "annihilate_without_pair": ("if (occupied == n) {", "if (occupied >= 1u) {"),
    "rate_p_not_p_times_1_minus_d": ("double scaled_a = p * (1.0 - d);", "double scaled_a = p;"),
    "phase_always_zero": ("return (uint32_t)(((uint64_t)out[0] * (uint64_t)L) >> 32);", "return 0u;"),
    "windows_cover_wrap": ("W = n_tup + 1u, K = L / W;", "W = n_tup + 1u, K = (L + n_tup) / W;"),
    "diffusion_swaps_a_c": ("uint8_t tmp = row[site[first]];\n        row[site[first]] = row[site[first + 1]];\n"
                            "        row[site[first + 1]] = tmp;",
                            "uint8_t tmp = row[site[0]];\n        row[site[0]] = row[site[n]];\n"
                            "        row[site[n]] = tmp;"),
    "time_floor_not_ceil": ("return (uint64_t)((num + K - 1) / K);", "return (uint64_t)(num / K);"),
    "pair_wrong_neighbour": ("pc += row[i] & row[(i + 1u) % jb->L];", "pc += row[i] & row[(i + 2u) % jb->L];"),
    # mistakes that only the n-tuple processes (R14) can show
    "tuple_annihilates_two_sites": ("for (uint32_t j = 0; j < n; ++j) row[site[first + j]] = 0;",
                                    "for (uint32_t j = 0; j < 2u; ++j) row[site[first + j]] = 0;"),
    "tuple_target_next_to_pair": ("const uint32_t target = o ? 0u : n;", "const uint32_t target = o ? 0u : 2u;"),
    # mistakes in the paper's own scheme (R13)
    "paper_draw_not_broadcast": ("if (dec && corr) {", "if (dec && ((words[m + n_dec] >> b) & 1u)) {"),
    "paper_fission_always_high": ("} else if ((fis >> b) & 1u) {", "} else if (fis | 1u) {"),
    "paper_diffusion_le": ("const int diffuse = u < t_d;", "const int diffuse = u <= t_d;"),
    "paper_site_per_workitem": ("(uint64_t)w * n_loc + istar;", "(uint64_t)w * n_loc + (istar + w) % n_loc;"),
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
    yield "paper_shared_site", lambda: TPS.test_same_local_site_in_every_workitem(mod, 4, 32)
    yield "paper_annihilation_law", lambda: TPS.test_first_step_annihilation_law(mod, 0.15, 2)
    yield "paper_diffusion_law", lambda: TPS.test_one_step_diffusion_law(mod, 0.25, 2)
    yield "paper_fission_sides", lambda: TPS.test_one_step_fission_sides(mod)
    for n in (3, 4):
        yield f"tuple{n}_bookkeeping", (lambda n=n: TU.test_bookkeeping_and_d1_conservation(mod, n))
        yield f"tuple{n}_closed_form", (lambda n=n: TU.test_p1_d0_first_substep_closed_form(mod, n, 61))
        yield f"tuple{n}_exact_chain", (lambda n=n: TU.test_schedule_oracle_matches_exact_chain(mod, n, 2 * n))


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
