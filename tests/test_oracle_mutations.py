"""Planted mistakes: the oracle's pins must catch them.

Each case writes a copy of ``oracle/ising_oracle.c`` with one plausible mistake
planted in it (a sign, a neighbour index, a parity test, a constant, a formula),
builds it into a temporary library, loads the oracle's Python wrapper on that
library and runs the pin tests named for the case on it.  At least one of them
must fail.  Mistakes that change only the random-number contract, which is a
definition and not a result, are not planted (no pin can tell one contract from
another).  CPU only; the mutants live in a temporary directory.
"""
import importlib.util
import os
import shutil

import pytest

import test_oracle_field as F
import test_oracle_philox as PH
import test_oracle_thresholds as TH
import test_oracle_update as U

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ising_oracle.c")
TC = 2.269185

# (name, text in the source, replacement, which occurrence, pins that must catch it)
MUTANTS = [
    ("energy change sign", "int dE_site = 2 * v * nsum;", "int dE_site = -2 * v * nsum;", 0,
     [lambda m: U.test_one_step_flip_frequencies_match_exact_probabilities(m, TC, 0, 6)]),
    ("right neighbour two sites away", "s[(uint64_t)r * L + (x + 1) % L]", "s[(uint64_t)r * L + (x + 2) % L]", 0,
     [U.test_one_step_dM_dE_bookkeeping_is_exact]),
    ("threshold exponent", "double v = floor(ldexp(exp(-dE / T), 32));", "double v = floor(ldexp(exp(-dE * T), 32));",
     0, [lambda m: TH.test_thresholds_match_60_digit_floor(m, 2.0)]),
    ("updated parity", "if (((x + y) & 1u) != p) continue;", "if (((x + y) & 1u) == p) continue;", 0,
     [lambda m: U.test_one_step_flip_frequencies_match_exact_probabilities(m, TC, 1, 6)]),
    ("energy bookkeeping sign", "dE += dE_site;", "dE -= dE_site;", 0,
     [U.test_one_step_dM_dE_bookkeeping_is_exact]),
    ("recount drops the vertical bonds", "e -= v * (s[y * L + xr] + s[yd * L + x]);", "e -= v * s[y * L + xr];", 0,
     [U.test_recount_closed_forms]),
    ("Binder cumulant factor", "out[6] = 1.0 - out[3] / (3.0 * out[2] * out[2]);",
     "out[6] = 1.0 - out[3] / (2.0 * out[2] * out[2]);", 0, [U.test_moments_closed_forms]),
    ("Philox Weyl constant", "#define PHILOX_WEYL_B 0xBB67AE85u", "#define PHILOX_WEYL_B 0xBB67AE84u", 0,
     [PH.test_philox_matches_triton_interpreter]),
    ("Philox word order", "uint32_t y2 = pa_hi ^ x3 ^ k1;", "uint32_t y2 = pa_hi ^ x1 ^ k1;", 0,
     [PH.test_philox_matches_triton_interpreter]),
    ("light-cone margin", "const uint64_t margin = 2 * k + 1;", "const uint64_t margin = k;", 0,
     [U.test_cold_tiled_counts_equal_whole_lattice_run]),
    ("field term sign", "double dE = 2.0 * (double)v * ((double)nsum + H);",
     "double dE = 2.0 * (double)v * ((double)nsum - H);", 0,
     [lambda m: F.test_one_step_flip_frequencies_in_a_field(m, TC, 0.3, 0, 6)]),
    ("field term without the spin", "double dE = 2.0 * (double)v * ((double)nsum + H);",
     "double dE = 2.0 * ((double)v * (double)nsum + H);", 0, [F.test_field_reversal_symmetry]),
    ("field bookkeeping", "dEb += 2 * v * nsum;", "dEb += 2 * nsum;", 0,
     [F.test_one_step_bookkeeping_and_recount_in_a_field]),
]


def _mutant(tmp_path, old, new, occurrence):
    src = open(SRC).read()
    pos = -1
    for _ in range(occurrence + 1):
        pos = src.index(old, pos + 1)
    mutated = src[:pos] + new + src[pos + len(old):]
    assert mutated != src
    d = tmp_path / "mutant"
    d.mkdir()
    (d / "ising_oracle.c").write_text(mutated)
    spec = importlib.util.spec_from_file_location("oracle_mutant_%d" % abs(hash((old, new))),
                                                  os.path.join(ROOT, "oracle", "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC = str(d / "ising_oracle.c")
    mod._LIB_PATH = str(d / "libising_oracle.so")
    mod._lib = None
    mod.build(force=True)
    return mod


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name,old,new,occurrence,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new, occurrence, pins):
    mod = _mutant(tmp_path, old, new, occurrence)
    caught = 0
    for pin in pins:
        try:
            pin(mod)
        except AssertionError:
            caught += 1
    assert caught > 0, "no pin caught the planted mistake: %s" % name


def test_unmutated_copy_passes_the_same_pins(tmp_path):
    """The harness itself: a copy with a no-op change passes every pin used above."""
    mod = _mutant(tmp_path, "#include <math.h>", "#include <math.h>\n", 0)
    for *_, pins in MUTANTS:
        for pin in pins:
            pin(mod)
