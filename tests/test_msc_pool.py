"""The paper's CPU multi-spin-coding program with a Boltzmann-pattern pool
(Sec. 4; oracle/msc_pool.c), the second CPU baseline.  It draws one pool
address per 32-spin word, so it is not bit-exact with the library or the
oracle; it is pinned here by the pool's bit statistics, by deterministic
limits, and by Onsager's exact magnetisation and energy far from T_c, where a
64 x 64 lattice is effectively infinite."""
import numpy as np
import pytest

from oracle import exact


@pytest.fixture(scope="module")
def msc():
    from oracle import msc

    msc.build()
    return msc


def _mean_err(x, nbins=20):
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nbins * nbins
    b = x[:n].reshape(nbins, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nbins)


@pytest.mark.parametrize("T", [0.8, 2.269185, 3.5])
def test_pool_bits_follow_the_encoding(msc, orc, T):
    """exp8 marks u < thr8, exp4 marks thr8 <= u < thr4: never both, and each
    bit is set with probability thr8 / 2^32 and (thr4 - thr8) / 2^32."""
    pool = msc.Pool(T, 1 << 16, seed=7)
    assert not np.any(pool.exp4 & pool.exp8)
    thr4, thr8 = orc.thresholds(T)
    nbits = pool.npool * 32
    for words, p in ((pool.exp8, thr8 / 2 ** 32), (pool.exp4, (thr4 - thr8) / 2 ** 32)):
        k = int(np.unpackbits(words.view(np.uint8)).sum())
        sd = np.sqrt(nbits * p * (1 - p))
        assert abs(k - nbits * p) <= 5 * sd + 1e-9, (k, nbits * p, sd)


def test_zero_temperature_limits(msc):
    L = 64
    pool = msc.Pool(0.01, 1 << 10)
    cold = msc.pack(np.ones((L, L), dtype=np.int8))
    M, E = msc.sweeps(cold, pool, 5, seed=3)
    assert np.all(M == L * L) and np.all(E == -2 * L * L)
    y, x = np.indices((L, L))
    neel = msc.pack(np.where((x + y) % 2 == 0, 1, -1).astype(np.int8))
    M, E = msc.sweeps(neel, pool, 1, seed=3)
    # step p = 0: every parity-0 site has four anti-aligned neighbours and flips
    assert M[0] == -L * L and E[0] == -2 * L * L
    assert np.all(msc.unpack(neel) == -1)


def test_pack_round_trip_and_recount(msc, orc):
    s = orc.init_hot(64, 5, 1)
    lat = msc.pack(s)
    assert np.array_equal(msc.unpack(lat), s)
    assert msc.recount(lat) == orc.recount(s)


@pytest.mark.parametrize("T,init,burn,n", [(1.5, "cold", 500, 6000), (3.5, "hot", 500, 6000)])
def test_onsager_far_from_tc(msc, orc, T, init, burn, n):
    """<|m|> (ordered phase) and the energy per spin against Onsager's exact
    infinite-lattice values, within 5 binned standard errors plus 1e-3."""
    L = 64
    N = L * L
    pool = msc.Pool(T, 1 << 20, seed=11)
    s = np.ones((L, L), dtype=np.int8) if init == "cold" else orc.init_hot(L, 4, 0)
    lat = msc.pack(s)
    M, E = msc.sweeps(lat, pool, n, seed=21)
    e, de = _mean_err(E[burn:] / N)
    assert abs(e - exact.onsager_u(T)) <= 5 * de + 1e-3, (e, de, exact.onsager_u(T))
    if T < 2.269185:
        m, dm = _mean_err(np.abs(M[burn:]) / N)
        assert abs(m - exact.onsager_m0(T)) <= 5 * dm + 1e-3, (m, dm, exact.onsager_m0(T))
    else:
        m2, dm2 = _mean_err((M[burn:] / N) ** 2)
        assert m2 < 0.01  # disordered: <m^2> ~ chi T / N
