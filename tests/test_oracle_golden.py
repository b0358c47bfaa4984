"""Oracle pins against stored values: the paper's printed numbers and the exact
references written by tests/golden/make_exact_refs.py (which calls only oracle.exact)."""
import json
import os

import pytest

from oracle import exact

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_paper_critical_temperature():
    pv = _load("paper_values.json")["critical_temperature"]
    assert round(exact.onsager_tc(), pv["digits"]) == pv["value"]


def test_exact_refs_reproduce():
    ref = _load("exact_refs.json")
    for T_s, vals in ref["4x4"].items():
        got = exact.enumerate_averages(4, float(T_s))
        for k, v in vals.items():
            assert got[k] == pytest.approx(v, rel=1e-13, abs=1e-15)
    assert ref["6x6_total_states"] == 2.0 ** 36


def test_transfer_matrix_agrees_with_enumeration_on_4x4():
    for T in (1.5, 2.269185, 3.5):
        a = exact.enumerate_averages(4, T)
        b = exact.transfer_averages(4, T)
        for k in a:
            assert a[k] == pytest.approx(b[k], rel=1e-12, abs=1e-14)


def test_6x6_low_temperature_limit():
    # T -> 0: only the two ground states (E = -2N, |m| = 1) survive
    d = exact.transfer_averages(6, 0.05)
    assert d["mean_e"] == pytest.approx(-2.0, abs=1e-12)
    assert d["mean_abs_m"] == pytest.approx(1.0, abs=1e-12)
    assert d["U4"] == pytest.approx(2.0 / 3.0, abs=1e-12)
