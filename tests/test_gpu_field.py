"""GPU parity of the field update (Sec. 3, Eq. 1 with H != 0) and of temperature
and field changes between calls (annealing), against the oracle, bit for bit.

Every lattice and every recorded M and E (E the bond energy) must equal the
oracle's.  Sizes span one block with idle threads (L = 64, 192), word counts per
row that are not a multiple of the warp (L = 192, 1088) and many blocks
(L = 1088, 4096); the fields cover every arrangement of the always-accepted
classes: |H| < 2, the boundaries H = +-2 and +-4 where a class has dE = 0, and
|H| > 4 where a spin against the field always flips.
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


def _pair(P, orc, L, T, H, seed, stream_id, nsweeps, word_bits, init="hot", buf=None):
    lat = P.Lattice(L, T, seed=seed, stream_id=stream_id, init=init, spins=buf, word_bits=word_bits, H=H)
    if init == "hot":
        s = orc.init_hot(L, seed, stream_id)
    elif init == "cold_down":
        s = orc.init_cold(L, -1)
    elif init == "cold_up":
        s = orc.init_cold(L, 1)
    else:
        s = np.ascontiguousarray(buf, dtype=np.int8)
    M, E = lat.sweep(nsweeps, 1, collect=True)
    Mo, Eo = orc.run_field(s, nsweeps, seed, stream_id, T, H, check=True)
    assert np.array_equal(M, Mo) and np.array_equal(E, Eo)
    assert np.array_equal(lat.spins(), s)
    return lat, s


@pytest.mark.parametrize("word_bits", [32, 64])
@pytest.mark.parametrize("L", [64, 192, 1088])
@pytest.mark.parametrize("H", [0.1, -0.37, 1.0])
def test_field_sweeps_bit_exact(P, orc, L, word_bits, H):
    _pair(P, orc, L, TC, H, seed=L + 7, stream_id=3, nsweeps=15, word_bits=word_bits)


@pytest.mark.parametrize("T,H", [(1.5, 2.0), (2.0, -2.0), (3.0, 4.0), (2.5, -4.0), (0.8, 5.5),
                                 (TC, -7.25), (50.0, 0.3), (0.05, 0.5), (2.0, 1e-9)])
def test_field_boundaries_and_limits_bit_exact(P, orc, T, H):
    _pair(P, orc, 256, T, H, seed=5, stream_id=0, nsweeps=20, word_bits=32)


@pytest.mark.parametrize("init", ["cold_up", "cold_down"])
def test_field_against_the_ordered_state(P, orc, init):
    # a field opposing the cold start drives the reversal
    _pair(P, orc, 320, 2.0, 0.25 if init == "cold_down" else -0.25, seed=12, stream_id=1,
          nsweeps=40, word_bits=64, init=init)


def test_field_larger_lattice_bit_exact(P, orc):
    _pair(P, orc, 4096, TC, 0.05, seed=77, stream_id=2, nsweeps=4, word_bits=32)


def test_strong_field_aligns_in_one_sweep(P):
    L = 512
    with P.Lattice(L, 0.5, init="cold_down", H=10.0) as lat:
        M, E = lat.sweep(3, 1, collect=True)
        assert list(M) == [L * L] * 3 and list(E) == [-2 * L * L] * 3
        assert np.all(lat.spins() == 1)


def test_field_reversal_symmetry_on_the_gpu(P):
    """(S, H) -> (-S, -H): the reversed start in the reversed field gives the
    reversed lattice and samples."""
    rng = np.random.default_rng(3)
    L = 256
    s0 = np.where(rng.random((L, L)) < 0.5, 1, -1).astype(np.int8)
    a = P.Lattice(L, 2.1, seed=4, spins=s0, H=0.6)
    b = P.Lattice(L, 2.1, seed=4, spins=(-s0).astype(np.int8), H=-0.6)
    Ma, Ea = a.sweep(25, 1, collect=True)
    Mb, Eb = b.sweep(25, 1, collect=True)
    assert np.array_equal(Ma, -Mb) and np.array_equal(Ea, Eb)
    assert np.array_equal(a.spins(), -b.spins())
    a.close()
    b.close()


def test_annealing_schedule_bit_exact(P, orc):
    """Temperature and field changed between calls (set_temperature, set_field),
    including switches between H = 0 (the zero-field kernel) and H != 0; the
    oracle applies the same schedule sweep by sweep."""
    L, seed, sid = 192, 31, 4
    schedule = [(3.5, 0.0, 5), (3.0, 0.0, 4), (2.6, 0.2, 6), (TC, 0.2, 3), (2.0, -0.1, 5),
                (1.5, 0.0, 4), (1.2, 3.0, 3), (1.2, 0.0, 2)]
    lat = P.Lattice(L, schedule[0][0], seed=seed, stream_id=sid, init="hot", word_bits=32)
    s = orc.init_hot(L, seed, sid)
    t = 0
    allM, allMo = [], []
    for T, H, n in schedule:
        lat.set_temperature(T)
        lat.set_field(H)
        assert (lat.T, lat.H) == (T, H)
        M, E = lat.sweep(n, 1, collect=True)
        if H == 0.0:
            thr4, thr8 = orc.thresholds(T)
            Mo, Eo = orc.run(s, n, seed, sid, thr4, thr8, t0=t)
        else:
            Mo, Eo = orc.run_field(s, n, seed, sid, T, H, t0=t)
        assert np.array_equal(M, Mo) and np.array_equal(E, Eo), (T, H)
        allM.append(M)
        allMo.append(Mo)
        t += n
    assert np.array_equal(lat.spins(), s)
    # the handle's sample history is the concatenation; moments use the last T
    Ms, _ = lat.samples()
    assert np.array_equal(Ms, np.concatenate(allMo))
    obs = lat.measure()
    assert obs["chi"] == pytest.approx(L * L * (obs["mean_m2"] - obs["mean_abs_m"] ** 2) / schedule[-1][0],
                                       rel=1e-12)
    lat.close()


def test_field_split_calls_and_checkpoint(P, orc, tmp_path):
    """Sweeps in a field split over calls and over a save/load equal one run."""
    L, T, H = 128, 2.4, -0.45
    a = P.Lattice(L, T, seed=8, H=H)
    a.sweep(7, 1)
    path = str(tmp_path / "f.npz")
    a.save(path)
    b = P.Lattice.load(path)
    assert b.H == H and b.T == T
    Mb, Eb = b.sweep(9, 1, collect=True)
    s = orc.init_hot(L, 8, 0)
    Mo, Eo = orc.run_field(s, 16, 8, 0, T, H)
    assert np.array_equal(Mb, Mo[7:]) and np.array_equal(Eb, Eo[7:])
    assert np.array_equal(b.spins(), s)
    a.close()
    b.close()


def test_batch_in_a_field_bit_exact(P, orc):
    """A persistent batch that mixes lattices in a field with zero-field ones, one
    of them over several CTAs with border exchange (L = 2048), against the
    oracle's field update lattice by lattice."""
    specs = [(64, 2.0, 0.3), (128, 2.4, 0.0), (256, 1.8, -1.0), (512, 3.0, 2.5), (2048, 2.269185, 0.1)]
    n, re = 6, 2
    lats = [P.Lattice(L, T, seed=40 + i, stream_id=i, init="hot", H=H) for i, (L, T, H) in enumerate(specs)]
    with P.Batch(lats, [n] * len(lats), re) as b:
        assert b.info()["strips"] > len(lats)  # the L = 2048 lattice is split into strips
        b.run(1)
    for i, ((L, T, H), lat) in enumerate(zip(specs, lats)):
        s = orc.init_hot(L, 40 + i, i)
        if H == 0.0:
            thr4, thr8 = orc.thresholds(T)
            Mo, Eo = orc.run(s, n, 40 + i, i, thr4, thr8)
        else:
            Mo, Eo = orc.run_field(s, n, 40 + i, i, T, H)
        M, E = lat.samples()
        assert np.array_equal(M, Mo[re - 1::re]) and np.array_equal(E, Eo[re - 1::re]), (L, H)
        assert np.array_equal(lat.spins(), s), (L, H)
        lat.close()


def test_server_in_a_field_equals_alone(P):
    """Served requests in a field give the same samples as the same lattice run alone."""
    reqs = [dict(L=64, T=2.0, H=0.4, n=30), dict(L=256, T=2.5, H=-0.2, n=20), dict(L=128, T=1.5, H=0.0, n=25),
            dict(L=512, T=3.0, H=1.7, n=12)]
    with P.Server(hbm_budget_bytes=1 << 26, epoch_sweeps=7, keep_samples=True) as srv:
        ids = [srv.submit(r["L"], r["T"], r["n"], seed=100 + i, record_every=1, tag=i, H=r["H"])
               for i, r in enumerate(reqs)]
        got = {}
        while len(got) < len(reqs):
            for res in srv.poll(wait_s=1.0):
                got[res["tag"]] = res
        for i, r in enumerate(reqs):
            assert got[i]["status"] == P.OK
            M, E = srv.samples(ids[i])
            with P.Lattice(r["L"], r["T"], seed=100 + i, init="hot", H=r["H"]) as lat:
                Ma, Ea = lat.sweep(r["n"], 1, collect=True)
            assert np.array_equal(M, Ma) and np.array_equal(E, Ea), r


def test_batch_keeps_the_field_it_was_made_with(P, orc):
    """A batch takes each lattice's field when it is made; set_field afterwards
    changes ising_sweep, not the batch's runs."""
    L, T = 128, 2.2
    lat = P.Lattice(L, T, seed=3, init="hot", H=0.5)
    with P.Batch([lat], [4], 1) as b:
        lat.set_field(0.0)
        b.run(1)
    s = orc.init_hot(L, 3, 0)
    orc.run_field(s, 4, 3, 0, T, 0.5)
    assert np.array_equal(lat.spins(), s)
    lat.close()


def test_set_temperature_validates(P):
    with P.Lattice(64, 2.0) as lat:
        for bad in (0.0, -1.0, float("nan"), float("inf")):
            with pytest.raises(P.IsingError):
                lat.set_temperature(bad)
        with pytest.raises(P.IsingError):
            lat.set_field(float("nan"))
        assert (lat.T, lat.H) == (2.0, 0.0)
