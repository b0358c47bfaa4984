"""Pins of the Metropolis thresholds thr(dE) = floor(2^32 exp(-dE/T)) (Sec. 3, Eq. 3).

The reference value is computed with 60-digit arithmetic (mpmath) from the same
FP64 temperature; the FP64 computation must give the same integer unless the
exact value lies within 1e-6 of an integer (then the FP64 rounding may pick
either side and the case is skipped).
"""
import math

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")


def _exact_floor(dE, T):
    with mpmath.workdps(60):
        v = mpmath.ldexp(mpmath.exp(-mpmath.mpf(dE) / mpmath.mpf(T)), 32)
        fl = mpmath.floor(v)
        return int(fl), float(v - fl)


@pytest.mark.parametrize("T", [0.5, 1.0, 1.5, 2.0, 2.20, 2.246493, 2.269185, 2.35, 3.5, 10.0, 1e3])
def test_thresholds_match_60_digit_floor(orc, T):
    t4, t8 = orc.thresholds(T)
    for dE, got in ((4, t4), (8, t8)):
        want, frac = _exact_floor(dE, T)
        if 1e-6 < frac < 1 - 1e-6:
            assert got == want, (T, dE, got, want)


def test_thresholds_random_temperatures(orc):
    rng = np.random.default_rng(3)
    for T in rng.uniform(0.3, 50.0, size=200):
        t4, t8 = orc.thresholds(float(T))
        for dE, got in ((4, t4), (8, t8)):
            want, frac = _exact_floor(dE, float(T))
            if 1e-6 < frac < 1 - 1e-6:
                assert got == want


def test_threshold_limits_and_ordering(orc):
    # T -> 0+: nothing with dE > 0 is ever accepted
    assert orc.thresholds(0.01) == (0, 0)
    # thr8 <= thr4, both decreasing as T falls; thr8 ~ thr4^2 / 2^32 (exp(-8/T) = exp(-4/T)^2)
    prev = (2 ** 32, 2 ** 32)
    for T in np.linspace(50.0, 0.2, 300):
        t4, t8 = orc.thresholds(float(T))
        assert t8 <= t4 <= prev[0] and t8 <= prev[1]
        assert abs(t8 - t4 * t4 / 2.0 ** 32) <= 2.0
        prev = (t4, t8)
    # a temperature so high that exp(-4/T) rounds to 1.0 is clamped to 2^32 - 1
    assert orc.thresholds(1e300) == (0xFFFFFFFF, 0xFFFFFFFF)


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan"), float("inf"), -float("inf")])
def test_threshold_rejects_bad_temperature(orc, bad):
    with pytest.raises(ValueError):
        orc.thresholds(bad)


def test_onsager_tc_matches_paper_value():
    # Sec. 1 quotes T_C ~ 2.269185 (Onsager); the oracle's closed form must round to it
    from oracle import exact

    assert round(exact.onsager_tc(), 6) == 2.269185
    assert math.isclose(exact.onsager_tc(), 2.0 / math.asinh(1.0), rel_tol=1e-15)
