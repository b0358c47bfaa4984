"""Pins of the oracle's update in a nonzero field H (Sec. 3, Eq. 1 keeps the term
-H sum_i S_i, which the paper then sets to zero).

Flipping S with neighbour sum n changes the energy by dE = 2 S (n + H).  Each
test checks the oracle against something it does not compute itself: the
zero-field update, thresholds in 60-digit arithmetic, real Metropolis
probabilities, exact Boltzmann averages in a field (4x4 brute force, 6x6
transfer matrix), the (S, H) -> (-S, -H) symmetry, and deterministic limits.
"""
import numpy as np
import pytest

from oracle import exact

TC = 2.269185


def _random_state(L, seed):
    rng = np.random.default_rng(seed)
    return np.where(rng.random((L, L)) < 0.5, 1, -1).astype(np.int8)


@pytest.mark.parametrize("L,T", [(8, 1.5), (32, TC), (64, 3.0)])
def test_zero_field_equals_zero_field_update(orc, L, T):
    """H = 0 reproduces the zero-field update (thr4 / thr8 of Sec. 3) bit for bit."""
    thr4, thr8 = orc.thresholds(T)
    a = orc.init_hot(L, seed=21, stream_id=2)
    b = a.copy()
    Ma, Ea = orc.run(a, 40, seed=21, stream_id=2, thr4=thr4, thr8=thr8)
    Mb, Eb = orc.run_field(b, 40, seed=21, stream_id=2, T=T, H=0.0)
    assert np.array_equal(a, b)
    assert np.array_equal(Ma, Mb) and np.array_equal(Ea, Eb)


def test_field_thresholds_against_60_digit_arithmetic(orc):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    two32 = mpmath.mpf(2) ** 32
    for T in (0.3, 1.0, 2.0, TC, 3.7, 40.0):
        for H in (0.0, 0.1, -0.37, 1.0, 2.0, -2.0, 3.5, 6.0, -9.25):
            thr, alw = orc.field_thresholds(T, H)
            for i, S in enumerate((-1, 1)):
                for c in range(5):
                    n = S * (4 - 2 * c)
                    dE = 2 * S * (n + mpmath.mpf(H))
                    k = 5 * i + c
                    if dE <= 0:
                        assert alw[k] and thr[k] == 0, (T, H, S, c)
                        continue
                    assert not alw[k]
                    x = two32 * mpmath.exp(-dE / mpmath.mpf(T))
                    want = min(int(mpmath.floor(x)), 2 ** 32 - 1)
                    if abs(x - mpmath.nint(x)) > 1e-6:   # away from an integer: exact
                        assert int(thr[k]) == want, (T, H, S, c)
                    else:
                        assert abs(int(thr[k]) - want) <= 1
            # (S, c, H) and (-S, c, -H) have the same energy change
            thr_m, alw_m = orc.field_thresholds(T, -H)
            assert np.array_equal(thr[:5], thr_m[5:]) and np.array_equal(alw[:5], alw_m[5:])


@pytest.mark.parametrize("T,H,p,L", [(TC, 0.3, 0, 6), (1.2, -0.8, 1, 6), (2.0, 2.0, 0, 8), (3.5, 5.0, 1, 4)])
def test_one_step_flip_frequencies_in_a_field(orc, T, H, p, L):
    """Over many seeds each site flips with min(1, exp(-dE/T)), dE = 2 S (n + H);
    sites of the other parity never flip."""
    s0 = _random_state(L, 101 + L + p)
    want = exact.metropolis_probabilities(s0, p, T, H)
    n = 20000
    counts = np.zeros((L, L))
    for seed in range(n):
        s = s0.copy()
        orc.half_sweep_field(s, t=9, p=p, seed=seed * 2654435761 + 7, stream_id=1, T=T, H=H)
        counts += s != s0
    freq = counts / n
    sigma = np.sqrt(np.maximum(want * (1 - want), 1e-12) / n)
    assert np.all(freq[want == 0.0] == 0.0)
    assert np.all(freq[want == 1.0] == 1.0)
    assert np.all(np.abs(freq - want) <= 5.5 * sigma + 1e-6)


def test_field_reversal_symmetry(orc):
    """(S, H) -> (-S, -H) leaves every energy change unchanged, so the chain from
    the reversed start in the reversed field is the reversed chain, bit for bit.
    A sign slip in the field term breaks this."""
    for L, T, H in ((16, 2.0, 0.4), (32, TC, -1.3), (24, 1.1, 3.0)):
        a = _random_state(L, L)
        b = (-a).astype(np.int8)
        Ma, Ea = orc.run_field(a, 30, seed=8, stream_id=0, T=T, H=H)
        Mb, Eb = orc.run_field(b, 30, seed=8, stream_id=0, T=T, H=-H)
        assert np.array_equal(a, -b)
        assert np.array_equal(Ma, -Mb) and np.array_equal(Ea, Eb)


def test_one_step_bookkeeping_and_recount_in_a_field(orc):
    for L, T, H in ((4, 1.5, 0.5), (6, TC, -0.25), (32, 3.0, 1.0), (64, TC, 2.0)):
        s = _random_state(L, 3 * L)
        M0, E0 = orc.recount(s)
        for t in range(3):
            for p in (0, 1):
                dM, dE = orc.half_sweep_field(s, t=t, p=p, seed=5, stream_id=0, T=T, H=H)
                M1, E1 = orc.recount(s)
                assert (M1 - M0, E1 - E0) == (dM, dE)
                M0, E0 = M1, E1
        orc.run_field(s, 100, seed=5, stream_id=0, T=T, H=H, t0=3, check=True)


def test_zero_temperature_limit_is_deterministic(orc):
    """At T -> 0+ a site flips iff S (n + H) <= 0 (for H = 0.5 never zero):
    written out here with numpy from the definition, without any random draw."""
    L, H = 16, 0.5
    s = _random_state(L, 77)
    for p in (0, 1):
        want = s.astype(np.int64)
        n = np.roll(want, 1, 0) + np.roll(want, -1, 0) + np.roll(want, 1, 1) + np.roll(want, -1, 1)
        y, x = np.indices((L, L))
        flip = (((x + y) & 1) == p) & (want * (n + H) <= 0)
        want = np.where(flip, -want, want).astype(np.int8)
        orc.half_sweep_field(s, t=0, p=p, seed=1, stream_id=0, T=1e-3, H=H)
        assert np.array_equal(s, want)


def test_strong_field_aligns_a_reversed_lattice_in_one_sweep(orc):
    """All -1 in H = 10: step A flips every black site (dE = -12), step B every
    white one (dE = -28); at T = 0.5 the aligned state is then frozen."""
    L = 32
    s = orc.init_cold(L, -1)
    M, E = orc.run_field(s, 5, seed=3, stream_id=0, T=0.5, H=10.0)
    assert np.all(s == 1)
    assert list(M) == [L * L] * 5 and list(E) == [-2 * L * L] * 5


@pytest.mark.parametrize("L,T,H,nsweeps", [(4, 2.0, 0.3, 400000), (4, TC, -0.1, 400000),
                                           (4, 3.0, 1.0, 300000), (6, 2.5, 0.2, 200000)])
def test_chain_averages_in_a_field_match_exact_boltzmann(orc, L, T, H, nsweeps):
    """Long chains in a field reproduce the exact averages of Eq. 1 with H != 0
    (brute force 4x4, transfer matrix 6x6) within 5 sigma, including the signed
    magnetisation, which a wrong sign of the field term reverses."""
    ref = exact.enumerate_averages(L, T, H) if L == 4 else exact.transfer_averages(L, T, H)
    s = orc.init_hot(L, seed=19)
    M, E = orc.run_field(s, nsweeps, seed=19, stream_id=0, T=T, H=H, check=False)
    burn = nsweeps // 50
    N = L * L
    m = M[burn:] / N
    e = E[burn:] / N
    for name, series in (("mean_m", m), ("mean_e", e), ("mean_abs_m", np.abs(m)), ("mean_m2", m * m)):
        b = series[: (len(series) // 200) * 200].reshape(200, -1).mean(axis=1)
        mu, err = b.mean(), b.std(ddof=1) / np.sqrt(200)
        assert abs(mu - ref[name]) < 5 * err + 1e-12, (name, mu, ref[name], err)
    assert np.sign(ref["mean_m"]) == np.sign(H)


def test_exact_field_references_agree():
    """Brute force and transfer matrix agree in a field; M -> -M symmetry under H -> -H."""
    for T, H in ((1.5, 0.2), (TC, -0.7), (3.5, 2.5)):
        a = exact.enumerate_averages(4, T, H)
        b = exact.transfer_averages(4, T, H)
        for k in a:
            assert a[k] == pytest.approx(b[k], rel=1e-12, abs=1e-14)
        c = exact.enumerate_averages(4, T, -H)
        assert c["mean_m"] == pytest.approx(-a["mean_m"], rel=1e-12)
        assert c["mean_e"] == pytest.approx(a["mean_e"], rel=1e-12)
