"""GPU parity: the CUDA path through the C ABI against the oracle, bit for bit.

Every lattice, every recorded M and E, and the FP64 moments (1e-12 relative)
must equal the oracle's on the same seeded inputs.  Sizes span several thread
items, word columns and the ragged cases of the launch (one word per row,
a word count per row that is not a multiple of the warp, rows per item at the
lattice edge).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TC = 2.269185


@pytest.fixture(scope="module")
def P():
    import paper_1007_3726_gb300 as P

    P.build()
    P.load()
    return P


def _oracle_start(orc, L, init, seed, stream_id, buf=None):
    if init == "hot":
        return orc.init_hot(L, seed, stream_id)
    if init == "cold_up":
        return orc.init_cold(L, 1)
    if init == "cold_down":
        return orc.init_cold(L, -1)
    return np.ascontiguousarray(buf, dtype=np.int8)


def _run_pair(P, orc, L, T, seed, stream_id, init, nsweeps, word_bits, record_every=1, buf=None):
    lat = P.Lattice(L, T, seed=seed, stream_id=stream_id, init=init, spins=buf, word_bits=word_bits)
    s = _oracle_start(orc, L, init, seed, stream_id, buf)
    assert np.array_equal(lat.spins(), s), "initial state"
    assert lat.recount() == orc.recount(s)
    M, E = lat.sweep(nsweeps, record_every, collect=True)
    thr4, thr8 = orc.thresholds(T)
    Mo, Eo = orc.run(s, nsweeps, seed, stream_id, thr4, thr8, check=True)
    sel = slice(record_every - 1, None, record_every)
    assert np.array_equal(M, Mo[sel]) and np.array_equal(E, Eo[sel])
    assert np.array_equal(lat.spins(), s), "final lattice"
    return lat, s, Mo, Eo


@pytest.mark.parametrize("word_bits", [32, 64])
@pytest.mark.parametrize("L", [64, 128, 320, 1088])
def test_hot_start_sweeps_bit_exact(P, orc, L, word_bits):
    _run_pair(P, orc, L, TC, seed=L + 3, stream_id=5, init="hot", nsweeps=12, word_bits=word_bits)


@pytest.mark.parametrize("T", [0.8, 1.5, 2.0, 3.5, 50.0])
def test_temperatures_bit_exact(P, orc, T):
    _run_pair(P, orc, 192, T, seed=11, stream_id=0, init="hot", nsweeps=20, word_bits=32)


@pytest.mark.parametrize("init", ["cold_up", "cold_down"])
def test_cold_starts_bit_exact(P, orc, init):
    _run_pair(P, orc, 256, 2.0, seed=2, stream_id=1, init=init, nsweeps=25, word_bits=64)


def test_user_buffer_start_bit_exact(P, orc):
    rng = np.random.default_rng(4)
    L = 128
    buf = np.where(rng.random((L, L)) < 0.3, 1, -1).astype(np.int8)
    _run_pair(P, orc, L, TC, seed=9, stream_id=2, init="buffer", nsweeps=15, word_bits=32, buf=buf)


def test_plain_method_L64_1000_sweeps(P, orc):
    """L=64, T=2.269185, cold start +1, seed 1, 1000 sweeps, M and E every sweep."""
    lat, s, Mo, Eo = _run_pair(P, orc, 64, 2.269185, seed=1, stream_id=0, init="cold_up",
                               nsweeps=1000, word_bits=0)
    d = lat.measure()
    ref = orc.moments(Mo, Eo, N=64 * 64, T=2.269185)
    for k in ("mean_m", "mean_abs_m", "mean_m2", "mean_m4", "mean_e", "mean_e2", "U4", "chi", "C"):
        assert d[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-300), k
    assert d["n_samples"] == 1000 and d["sweeps_done"] == 1000
    assert (d["M"], d["E"]) == (int(Mo[-1]), int(Eo[-1]))
    # with the first 200 samples dropped as equilibration
    d2 = lat.measure(first_sample=200)
    ref2 = orc.moments(Mo, Eo, N=64 * 64, T=2.269185, burn=200)
    assert d2["n_samples"] == 800
    for k in ("mean_abs_m", "mean_m2", "mean_m4", "mean_e", "U4", "chi", "C"):
        assert d2[k] == pytest.approx(ref2[k], rel=1e-12, abs=1e-300), k


def test_split_calls_and_record_every_are_invariant(P, orc):
    L, T = 256, TC
    a = P.Lattice(L, T, seed=77, stream_id=3, init="hot")
    Ma, Ea = a.sweep(60, 3, collect=True)
    b = P.Lattice(L, T, seed=77, stream_id=3, init="hot")
    parts = [b.sweep(n, 3, collect=True) for n in (7, 13, 1, 39)]
    Mb = np.concatenate([p[0] for p in parts])
    Eb = np.concatenate([p[1] for p in parts])
    assert np.array_equal(Ma, Mb) and np.array_equal(Ea, Eb)
    assert np.array_equal(a.spins(), b.spins())
    # an asynchronous call followed by measure sees the same samples
    c = P.Lattice(L, T, seed=77, stream_id=3, init="hot")
    c.sweep(25, 3)
    c.sweep(35, 3)
    dc, da = c.measure(), a.measure()
    assert dc == da
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_hot(L, 77, 3)
    Mo, Eo = orc.run(s, 60, 77, 3, thr4, thr8)
    assert np.array_equal(Ma, Mo[2::3]) and np.array_equal(Ea, Eo[2::3])


def test_word_widths_agree(P):
    L = 1024
    a = P.Lattice(L, 2.1, seed=5, init="hot", word_bits=32)
    b = P.Lattice(L, 2.1, seed=5, init="hot", word_bits=64)
    Ma, Ea = a.sweep(40, 1, collect=True)
    Mb, Eb = b.sweep(40, 1, collect=True)
    assert np.array_equal(Ma, Mb) and np.array_equal(Ea, Eb)
    pa, pb = a.packed(), b.packed()
    assert pa.tobytes() == pb.tobytes()  # little-endian: the same bit string


def test_packed_start_round_trip(P, orc):
    L = 256
    a = P.Lattice(L, TC, seed=8, init="hot", word_bits=64)
    a.sweep(3)
    pk = a.packed()
    b = P.Lattice(L, TC, seed=8, init="packed", packed=pk, word_bits=64)
    assert np.array_equal(a.spins(), b.spins())


def test_neel_start_low_temperature(P):
    L = 256
    y, x = np.indices((L, L))
    neel = np.where((x + y) % 2 == 0, 1, -1).astype(np.int8)
    lat = P.Lattice(L, 0.01, seed=123, spins=neel)
    M, E = lat.sweep(1, 1, collect=True)
    assert M[0] == -L * L and E[0] == -2 * L * L
    assert np.all(lat.spins() == -1)


def test_zero_temperature_frozen_and_flip_symmetry(P):
    L = 512
    up = P.Lattice(L, 0.01, seed=1, init="cold_up")
    M, E = up.sweep(10, 1, collect=True)
    assert np.all(M == L * L) and np.all(E == -2 * L * L)
    a = P.Lattice(L, TC, seed=3, init="cold_up", word_bits=32)
    b = P.Lattice(L, TC, seed=3, init="cold_down", word_bits=32)
    Ma, Ea = a.sweep(30, 1, collect=True)
    Mb, Eb = b.sweep(30, 1, collect=True)
    assert np.array_equal(Ma, -Mb) and np.array_equal(Ea, Eb)
    assert np.array_equal(a.spins(), -b.spins())


def test_fused_counts_equal_recount(P):
    for L, wb in ((448, 32), (704, 64)):
        lat = P.Lattice(L, 2.3, seed=L, init="hot", word_bits=wb)
        for n in (1, 5, 17):
            lat.sweep(n, 0)
            d = lat.measure()
            assert (d["M"], d["E"]) == lat.recount()


def test_large_lattice_L32768(P, orc):
    """L=32768 (2^30 spins, 32-bit words), hot start seed 7, T=2.269185, 1000 sweeps,
    in the launch configuration the benchmark times.  Checked against the oracle:
    the whole initial state; M and E after every one of the first 100 sweeps and
    the whole lattice at sweep 100 (oracle on the whole lattice, about 75 s of
    host CPU); and a 2048-row strip at sweep 1000, evolved by the oracle from its
    own sweep-100 lattice in a light cone (900 sweeps need 1801 rows of margin on
    each side).  The fused counts of the last sweep equal a GPU recount."""
    L, T, seed = 32768, 2.269185, 7
    thr4, thr8 = orc.thresholds(T)
    lat = P.Lattice(L, T, seed=seed, init="hot", word_bits=32)
    cfg, _ = lat.autotune(reps=3)  # as bench.py does before it times
    assert cfg == lat.launch
    s = orc.init_hot(L, seed)
    assert np.array_equal(lat.spins(), s)
    M, E = lat.sweep(100, 1, collect=True)
    Mo, Eo = orc.run(s, 100, seed, 0, thr4, thr8, check=False)
    assert np.array_equal(M, Mo) and np.array_equal(E, Eo)
    assert np.array_equal(lat.spins(), s)
    row0, rows, k = 20000, 2048, 900
    margin = 2 * k + 1
    win = np.ascontiguousarray(s[row0 - margin:row0 + rows + margin])
    del s
    lat.sweep(k, 1)
    orc.run_window(win, L, row0 - margin, k, seed, 0, thr4, thr8, t0=100)
    got = lat.spins(row0, rows)
    assert np.array_equal(win[margin:margin + rows], got)
    d = lat.measure()
    assert d["sweeps_done"] == 1000 and d["n_samples"] == 1000
    assert (d["M"], d["E"]) == lat.recount()


def test_every_launch_configuration_is_bit_exact(P, orc):
    """Processing width, register cap, block size, rows per item and grid change
    only the speed: every candidate must reproduce the oracle bit for bit."""
    L, T, seed, sid, n = 320, TC, 91, 2, 3
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_hot(L, seed, sid)
    Mo, Eo = orc.run(s, n, seed, sid, thr4, thr8)
    cands = P.ising_launch_candidates(L)
    assert len(cands) >= 60
    extra = [dict(cands[0], grid=1), dict(cands[-1], grid=3), dict(cands[5], grid=7)]
    for cfg in cands + extra:
        lat = P.Lattice(L, T, seed=seed, stream_id=sid, init="hot", word_bits=32)
        lat.set_launch(**cfg)
        M, E = lat.sweep(n, 1, collect=True)
        assert np.array_equal(M, Mo) and np.array_equal(E, Eo), cfg
        assert np.array_equal(lat.spins(), s), cfg
        lat.close()


def test_grid_stride_on_a_wider_lattice(P, orc):
    L, T, seed, n = 2048, 2.2, 5, 4
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_hot(L, seed)
    Mo, Eo = orc.run(s, n, seed, 0, thr4, thr8)
    for cfg in ({"proc_bits": 32, "regcap": 0, "block": 128, "rows_per_item": 16, "grid": 5},
                {"proc_bits": 64, "regcap": 2, "block": 512, "rows_per_item": 2, "grid": 0},
                {"proc_bits": 64, "regcap": 1, "block": 256, "rows_per_item": 32, "grid": 152}):
        lat = P.Lattice(L, T, seed=seed, init="hot", word_bits=64)
        lat.set_launch(**cfg)
        M, E = lat.sweep(n, 1, collect=True)
        assert np.array_equal(M, Mo) and np.array_equal(E, Eo), cfg
        assert np.array_equal(lat.spins(), s), cfg


def test_autotune_keeps_the_lattice_and_the_results(P, orc):
    L, T, seed = 1024, TC, 13
    lat = P.Lattice(L, T, seed=seed, init="hot")
    lat.sweep(2, 1)
    before = lat.spins()
    cfg, us = lat.autotune(reps=1)
    assert cfg in P.ising_launch_candidates(L) and us > 0
    assert lat.launch == cfg
    assert np.array_equal(lat.spins(), before)
    M, E = lat.sweep(3, 1, collect=True)
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_hot(L, seed)
    Mo, Eo = orc.run(s, 5, seed, 0, thr4, thr8)
    assert np.array_equal(M, Mo[2:]) and np.array_equal(E, Eo[2:])
    assert np.array_equal(lat.spins(), s)
    # a later handle of the same size starts from the tuned configuration
    assert P.Lattice(L, 3.0, seed=1).launch == cfg


def test_invalid_launch_configurations_are_rejected(P):
    lat = P.Lattice(192, 2.0, seed=1)
    for bad in ({"proc_bits": 48}, {"regcap": 3}, {"block": 96}, {"rows_per_item": 5},
                {"rows_per_item": 128}, {"grid": 2 ** 24}):
        with pytest.raises(P.IsingError):
            lat.set_launch(**bad)
