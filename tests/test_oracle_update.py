"""Pins of the oracle's checkerboard Metropolis update (Sec. 3, Sec. 4).

Each test checks the oracle against something it does not compute itself:
exact flip probabilities of one checkerboard step, deterministic limits
(T -> 0+, the Neel start), symmetries, a full recount, and the light-cone
property of the local update.
"""
import numpy as np
import pytest

from oracle import exact

TC = 2.269185


def _random_state(L, seed):
    rng = np.random.default_rng(seed)
    return np.where(rng.random((L, L)) < 0.5, 1, -1).astype(np.int8)


@pytest.mark.parametrize("T,p,L", [(TC, 0, 6), (TC, 1, 6), (1.2, 0, 8), (3.5, 1, 4)])
def test_one_step_flip_frequencies_match_exact_probabilities(orc, T, p, L):
    """Over many independent seeds, every site flips with the exact probability
    1 (dE <= 0), thr4/2^32 (dE = 4) or thr8/2^32 (dE = 8), and sites of the other
    parity never flip (Sec. 3 acceptance and checkerboard rule)."""
    thr4, thr8 = orc.thresholds(T)
    s0 = _random_state(L, 11 + L + p)
    want = exact.flip_probabilities(s0, p, thr4, thr8)
    n = 20000
    counts = np.zeros((L, L))
    for seed in range(n):
        s = s0.copy()
        orc.half_sweep(s, t=5, p=p, seed=seed * 2654435761 + 1, stream_id=3, thr4=thr4, thr8=thr8)
        counts += s != s0
    freq = counts / n
    sigma = np.sqrt(np.maximum(want * (1 - want), 1e-12) / n)
    assert np.all(freq[want == 0.0] == 0.0)
    assert np.all(freq[want == 1.0] == 1.0)
    assert np.all(np.abs(freq - want) <= 5.5 * sigma + 1e-12)


def test_one_step_dM_dE_bookkeeping_is_exact(orc):
    thr4, thr8 = orc.thresholds(TC)
    for L in (4, 6, 10, 64):
        s = _random_state(L, L)
        M0, E0 = orc.recount(s)
        for t in range(3):
            for p in (0, 1):
                dM, dE = orc.half_sweep(s, t=t, p=p, seed=99, stream_id=0, thr4=thr4, thr8=thr8)
                M1, E1 = orc.recount(s)
                assert (M1 - M0, E1 - E0) == (dM, dE)
                M0, E0 = M1, E1


def test_incremental_equals_recount_every_sweep(orc):
    for L, T in ((4, 1.5), (8, TC), (32, 3.0), (64, TC)):
        thr4, thr8 = orc.thresholds(T)
        s = orc.init_hot(L, seed=5, stream_id=1)
        orc.run(s, 200, seed=5, stream_id=1, thr4=thr4, thr8=thr8, check=True)


def test_recount_closed_forms(orc):
    # all +1: M = N, E = -2N; checkerboard (Neel): M = 0, E = +2N; stripes: E = 0
    L = 8
    up = orc.init_cold(L, 1)
    assert orc.recount(up) == (L * L, -2 * L * L)
    assert orc.recount(orc.init_cold(L, -1)) == (-L * L, -2 * L * L)
    y, x = np.indices((L, L))
    neel = np.where((x + y) % 2 == 0, 1, -1).astype(np.int8)
    assert orc.recount(neel) == (0, 2 * L * L)
    stripes = np.where(x % 2 == 0, 1, -1).astype(np.int8)
    assert orc.recount(stripes) == (0, 0)


def test_zero_temperature_cold_start_is_frozen(orc):
    thr4, thr8 = orc.thresholds(0.01)
    assert (thr4, thr8) == (0, 0)
    s = orc.init_cold(16, 1)
    M, E = orc.run(s, 20, seed=1, stream_id=0, thr4=thr4, thr8=thr8)
    assert np.all(s == 1) and np.all(M == 256) and np.all(E == -512)


@pytest.mark.parametrize("seed", [0, 1, 12345, 2 ** 64 - 1])
def test_neel_start_at_low_temperature(orc, seed):
    """Step A (black, p = 0) of a Neel state: every black site has four
    anti-aligned neighbours (dE = -8) and flips, giving all -1; in step B every
    site has dE = +8 and thr8 = 0 never accepts.  So M = -N, E = -2N."""
    L = 12
    thr4, thr8 = orc.thresholds(0.01)
    y, x = np.indices((L, L))
    s = np.where((x + y) % 2 == 0, 1, -1).astype(np.int8)
    M, E = orc.run(s, 1, seed=seed, stream_id=0, thr4=thr4, thr8=thr8)
    assert np.all(s == -1) and M[0] == -L * L and E[0] == -2 * L * L


def test_global_spin_flip_symmetry(orc):
    """The random draws and thresholds do not depend on the sign of the spins,
    so the all -1 start is the mirror image of the all +1 start."""
    L, T = 16, TC
    thr4, thr8 = orc.thresholds(T)
    a = orc.init_cold(L, 1)
    b = orc.init_cold(L, -1)
    Ma, Ea = orc.run(a, 60, seed=3, stream_id=2, thr4=thr4, thr8=thr8)
    Mb, Eb = orc.run(b, 60, seed=3, stream_id=2, thr4=thr4, thr8=thr8)
    assert np.array_equal(a, -b) and np.array_equal(Ma, -Mb) and np.array_equal(Ea, Eb)
    h = orc.init_hot(L, seed=8)
    hm = (-h).astype(np.int8)
    Mh, Eh = orc.run(h, 30, seed=4, stream_id=0, thr4=thr4, thr8=thr8)
    Mm, Em = orc.run(hm, 30, seed=4, stream_id=0, thr4=thr4, thr8=thr8)
    assert np.array_equal(h, -hm) and np.array_equal(Mh, -Mm) and np.array_equal(Eh, Em)


def test_streams_and_seeds_give_different_chains(orc):
    L = 16
    thr4, thr8 = orc.thresholds(TC)
    runs = []
    for seed, stream in ((1, 0), (2, 0), (1, 1)):
        s = orc.init_cold(L, 1)
        orc.run(s, 10, seed=seed, stream_id=stream, thr4=thr4, thr8=thr8)
        runs.append(s)
    assert not np.array_equal(runs[0], runs[1]) and not np.array_equal(runs[0], runs[2])


def test_light_cone_window_matches_full_lattice(orc):
    """A window of rows updated with fixed edge rows agrees with the periodic
    lattice on the rows the edges have not reached (the update is local)."""
    L, T, k = 64, TC, 3
    thr4, thr8 = orc.thresholds(T)
    full = orc.init_hot(L, seed=21, stream_id=4)
    start = full.copy()
    orc.run(full, k, seed=21, stream_id=4, thr4=thr4, thr8=thr8, t0=7)
    for row0, nrows in ((10, 20), (50, 30), (0, 2 * 2 * k + 1)):
        rows = [(row0 + r) % L for r in range(nrows)]
        w = np.ascontiguousarray(start[rows])
        orc.run_window(w, L, row0, k, seed=21, stream_id=4, thr4=thr4, thr8=thr8, t0=7)
        inner = slice(2 * k, nrows - 2 * k)
        assert np.array_equal(w[inner], full[rows][inner])


def test_hot_start_is_fair_and_windows_agree(orc):
    L = 512
    s = orc.init_hot(L, seed=7)
    N = L * L
    plus = int((s == 1).sum())
    assert abs(plus - N / 2) < 5 * np.sqrt(N / 4)
    # neighbouring sites uncorrelated
    c = float((s[:, :-1].astype(np.int64) * s[:, 1:]).mean())
    assert abs(c) < 5 / np.sqrt(N)
    # a window of rows equals the same rows of the whole lattice
    w = orc.init_hot(L, seed=7, row0=500, nrows=30)
    assert np.array_equal(w, s[[(500 + r) % L for r in range(30)]])
    # another stream is another lattice
    assert not np.array_equal(orc.init_hot(L, seed=7, stream_id=1), s)


def _binned_mean(x, nbins=200):
    x = np.asarray(x, dtype=np.float64)
    n = (len(x) // nbins) * nbins
    b = x[:n].reshape(nbins, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nbins)


@pytest.mark.parametrize("L,T,nsweeps", [(4, 1.5, 400000), (4, TC, 400000), (4, 3.5, 400000),
                                         (6, TC, 200000), (6, 2.0, 200000)])
def test_chain_averages_match_exact_boltzmann(orc, L, T, nsweeps):
    """Long oracle chains reproduce the exact Boltzmann averages of Eq. 1
    (brute-force enumeration for 4x4, transfer matrix for 6x6) within 5 sigma."""
    ref = exact.enumerate_averages(L, T) if L == 4 else exact.transfer_averages(L, T)
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_hot(L, seed=17)
    M, E = orc.run(s, nsweeps, seed=17, stream_id=0, thr4=thr4, thr8=thr8, check=False)
    burn = nsweeps // 50
    N = L * L
    m = M[burn:] / N
    e = E[burn:] / N
    for name, series in (("mean_e", e), ("mean_abs_m", np.abs(m)), ("mean_m2", m * m),
                         ("mean_m4", m ** 4)):
        mu, err = _binned_mean(series)
        assert abs(mu - ref[name]) < 5 * err + 1e-12, (name, mu, ref[name], err)


def test_moments_closed_forms(orc):
    N = 100
    # |M| constant = N/2: <m^2> = 1/4, <m^4> = 1/16, U4 = 2/3, chi = 0
    M = np.array([50, -50, 50, 50, -50, 50], dtype=np.int64)
    E = np.array([-100, -60, -100, -20, -60, -100], dtype=np.int64)
    d = orc.moments(M, E, N=N, T=2.0)
    assert d["n_samples"] == 6
    assert d["mean_m"] == pytest.approx(1 / 6 * 0.5 * 2, rel=1e-15)
    assert d["mean_abs_m"] == 0.5 and d["mean_m2"] == 0.25 and d["mean_m4"] == 0.0625
    assert d["U4"] == pytest.approx(2 / 3, rel=1e-15) and d["chi"] == 0.0
    e = E / N
    assert d["mean_e"] == pytest.approx(e.mean(), rel=1e-15)
    assert d["C"] == pytest.approx(N * (np.mean(e * e) - e.mean() ** 2) / 4.0, rel=1e-12)
    # burn-in drops leading samples
    d2 = orc.moments(M, E, N=N, T=2.0, burn=4)
    assert d2["n_samples"] == 2 and d2["mean_m"] == 0.0
    # Gaussian magnetisation: U4 -> 0
    rng = np.random.default_rng(0)
    Mg = np.round(rng.normal(0, 1e6, size=200000)).astype(np.int64)
    dg = orc.moments(Mg, np.zeros_like(Mg), N=10 ** 8, T=1.0)
    assert abs(dg["U4"]) < 0.02


def test_onsager_closed_forms_against_finite_lattices():
    """The infinite-lattice energy closed form is approached by the exact 6x6
    lattice deep in the ordered phase, and equals -sqrt(2) at T_c."""
    assert exact.onsager_u(exact.onsager_tc() * (1 - 1e-7)) == pytest.approx(-np.sqrt(2), abs=1e-5)
    for T in (1.0, 1.3):
        u6 = exact.transfer_averages(6, T)["mean_e"]
        assert abs(u6 - exact.onsager_u(T)) < 2e-3
        m6 = exact.transfer_averages(6, T)["mean_abs_m"]
        assert abs(m6 - exact.onsager_m0(T)) < 5e-3
    assert exact.onsager_m0(3.0) == 0.0


def test_cold_tiled_counts_equal_whole_lattice_run(orc):
    """The tile-by-tile light-cone counts equal a run of the whole lattice."""
    for L, T, k, tile in ((64, 2.0, 3, 16), (128, TC, 4, 64), (96, 3.0, 2, 32)):
        thr4, thr8 = orc.thresholds(T)
        for up in (True, False):
            s = orc.init_cold(L, 1 if up else -1)
            M, E = orc.run(s, k, seed=5, stream_id=3, thr4=thr4, thr8=thr8)
            Mt, Et = orc.cold_tiled_counts(L, k, 5, 3, thr4, thr8, up=up, tile_rows=tile)
            assert np.array_equal(M, Mt) and np.array_equal(E, Et)
