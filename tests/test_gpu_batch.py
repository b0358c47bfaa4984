"""The persistent multi-lattice launch against the one-lattice path and the oracle.

A batch moves work between CTAs and in time, never changes the arithmetic: every
handle's samples, final M/E and lattice must equal what ising_sweep gives on an
identical handle, bit for bit, for uneven lattice sizes, sweeps, temperatures,
storage widths, strip counts (lattices split over many CTAs exchange border
rows), repeated runs and CUDA-graph replay.
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


def _spec(L, T, seed, sid, init="hot", wb=0):
    return dict(L=L, T=T, seed=seed, stream_id=sid, init=init, word_bits=wb)


def _make(P, specs):
    return [P.Lattice(**sp) for sp in specs]


def _reference(P, specs, sweeps, record_every, runs=1):
    out = []
    for sp, n in zip(specs, sweeps):
        lat = P.Lattice(**sp)
        M, E = lat.sweep(n * runs, record_every, collect=True)
        out.append((M, E, lat.spins(), lat.measure()))
        lat.close()
    return out


def _check(P, lats, ref):
    for lat, (M, E, s, d) in zip(lats, ref):
        got = lat.measure()
        assert got["sweeps_done"] == d["sweeps_done"]
        assert (got["M"], got["E"]) == (d["M"], d["E"])
        assert got["n_samples"] == d["n_samples"]
        assert got == d
        assert np.array_equal(lat.spins(), s)


SPECS = [_spec(64, TC, 1, 0, "cold_up"), _spec(128, 1.5, 2, 1), _spec(256, 2.2, 3, 2, wb=64),
         _spec(320, 3.5, 4, 3), _spec(512, TC, 5, 4, wb=32), _spec(1024, 2.0, 6, 5),
         _spec(2048, 2.3, 7, 6, wb=64), _spec(192, 0.8, 8, 7, "cold_down")]


@pytest.mark.parametrize("record_every", [1, 3])
def test_batch_equals_plain_uneven_sizes(P, record_every):
    sweeps = [9, 4, 7, 11, 5, 6, 3, 8]
    ref = _reference(P, SPECS, sweeps, record_every)
    lats = _make(P, SPECS)
    P.ising_sweep_batch(lats, sweeps, record_every)
    _check(P, lats, ref)


@pytest.mark.parametrize("opts", [dict(ctas_per_sm=4), dict(ctas_per_sm=1, block=256),
                                  dict(ctas_per_sm=3, rows_per_item=1, insert=2),
                                  dict(ctas_per_sm=2, rows_per_item=16, insert=1)])
def test_batch_options_and_strip_splits(P, opts):
    # with 4 CTAs per SM the L=2048 and L=4096 lattices are split over many CTAs
    specs = SPECS[:6] + [_spec(4096, TC, 9, 8), _spec(2048, 2.3, 7, 6, wb=64)]
    sweeps = [6, 6, 5, 4, 6, 5, 6, 7]
    ref = _reference(P, specs, sweeps, 2)
    lats = _make(P, specs)
    with P.Batch(lats, sweeps, 2, **opts) as b:
        info = b.info()
        assert info["strips"] >= len(specs)
        b.run(1)
    _check(P, lats, ref)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_repeated_runs(P, use_graph):
    specs = SPECS[:7]
    sweeps = [5, 4, 3, 6, 2, 3, 4]
    ref = _reference(P, specs, sweeps, 4, runs=3)
    lats = _make(P, specs)
    with P.Batch(lats, sweeps, 4, use_graph=use_graph) as b:
        b.run(2)
        b.run(1)
    _check(P, lats, ref)


def test_batch_after_plain_sweeps_and_oracle(P, orc):
    """A handle moved between the two paths keeps one trajectory."""
    L, T, seed, sid = 512, TC, 41, 9
    lat = P.Lattice(L, T, seed=seed, stream_id=sid, init="hot")
    lat.sweep(3, 1)
    P.ising_sweep_batch([lat], [4], 1)
    lat.sweep(2, 1)
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_hot(L, seed, sid)
    Mo, Eo = orc.run(s, 9, seed, sid, thr4, thr8)
    d = lat.measure()
    assert d["n_samples"] == 9 and (d["M"], d["E"]) == (int(Mo[-1]), int(Eo[-1]))
    assert np.array_equal(lat.spins(), s)
    ref = orc.moments(Mo, Eo, N=L * L, T=T)
    assert d["U4"] == pytest.approx(ref["U4"], rel=1e-12)


def test_plain_method_L64_in_one_launch(P, orc):
    """L=64, T=2.269185, cold start, seed 1, 1000 sweeps, M/E every sweep: one
    persistent launch (one CTA keeps the lattice in shared memory)."""
    lat = P.Lattice(64, 2.269185, seed=1, init="cold_up")
    with P.Batch([lat], [1000], 1) as b:
        assert b.info()["grid"] == 1
        b.run(1)
    thr4, thr8 = orc.thresholds(2.269185)
    s = orc.init_cold(64, 1)
    Mo, Eo = orc.run(s, 1000, 1, 0, thr4, thr8)
    d = lat.measure()
    ref = orc.moments(Mo, Eo, N=64 * 64, T=2.269185)
    for k in ("mean_m", "mean_abs_m", "mean_m2", "mean_m4", "mean_e", "mean_e2", "U4", "chi", "C"):
        assert d[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-300), k
    assert np.array_equal(lat.spins(), s)


def test_finite_size_scaling_batch_shape(P):
    """The 128-lattice shape (L in {256, 512, 1024, 2048} x 32 temperatures in
    [2.20, 2.35], hot starts, seed 3, stream 32 * iL + iT), 20 sweeps with a sample
    every 10, equals 128 one-lattice runs."""
    Ls = (256, 512, 1024, 2048)
    temps = [2.20 + i * 0.15 / 31 for i in range(32)]
    specs = [_spec(L, T, 3, 32 * iL + iT) for iL, L in enumerate(Ls) for iT, T in enumerate(temps)]
    sweeps = [20] * len(specs)
    ref = _reference(P, specs, sweeps, 10)
    lats = _make(P, specs)
    with P.Batch(lats, sweeps, 10, use_graph=True) as b:
        b.run(1)
    _check(P, lats, ref)


def test_batch_wait_limit_reports_timeout(P):
    """A strip that never announces its steps (a flag nothing sets): its
    neighbours' bounded waits run out, the launch returns, the host sees
    ISING_ERR_TIMEOUT and the handles refuse further work; the GPU stays usable."""
    lat = P.Lattice(4096, TC, seed=1, init="hot")
    other = P.Lattice(256, TC, seed=2, init="hot")
    with P.Batch([lat, other], [3, 3], 1, ctas_per_sm=4, wait_ms=50.0, hold_strip=1) as b:
        assert b.info()["strips"] > 2
        with pytest.raises(P.IsingError) as ei:
            b.run(1)
        assert ei.value.status == P.ERR_TIMEOUT
    with pytest.raises(P.IsingError) as ei:
        lat.sweep(1)
    assert ei.value.status == P.ERR_STATE
    # a fresh handle still works
    fresh = P.Lattice(256, TC, seed=2, init="hot")
    fresh.sweep(2, 1)
    assert fresh.measure()["sweeps_done"] == 2


def test_batch_rejects_bad_input(P):
    a = P.Lattice(256, 2.0, seed=1)
    with pytest.raises(P.IsingError):
        P.ising_sweep_batch([a, a], [1, 1], 0)
    with pytest.raises(P.IsingError):
        P.ising_sweep_batch([a], [0], 0)
    with pytest.raises(P.IsingError):
        P.Batch([a], [1], 0, block=1024)


def test_batch_tune_restores_lattices_and_results_stay_exact(P):
    specs = SPECS[:7]
    sweeps = [5, 4, 3, 6, 2, 3, 4]
    ref = _reference(P, specs, sweeps, 1)
    lats = _make(P, specs)
    before = [l.spins() for l in lats]
    opts, ms = P.ising_batch_tune(lats, sweeps, 4)
    assert ms > 0 and opts["block"] in (256, 512)
    for l, s0 in zip(lats, before):
        assert np.array_equal(l.spins(), s0)
        assert l.measure()["sweeps_done"] == 0
    with P.Batch(lats, sweeps, 1, **opts) as b:
        b.run(1)
    _check(P, lats, ref)


def test_samples_round_trip(P, orc):
    L, T = 128, 2.4
    lat = P.Lattice(L, T, seed=4, init="hot")
    lat.sweep(30, 2)
    M, E = lat.samples()
    s = orc.init_hot(L, 4)
    thr4, thr8 = orc.thresholds(T)
    Mo, Eo = orc.run(s, 30, 4, 0, thr4, thr8)
    assert np.array_equal(M, Mo[1::2]) and np.array_equal(E, Eo[1::2])
    M2, E2 = lat.samples(first=10, count=3)
    assert np.array_equal(M2, M[10:13]) and np.array_equal(E2, E[10:13])


def test_binder_crossing_small_lattices(P):
    """The paper's correctness test in miniature: U4 curves of L = 64 and 128
    cross near Onsager's T_c."""
    import math

    from paper_1007_3726_gb300 import fss

    res = fss.run_fss(Ls=(64, 128), temps=np.linspace(2.20, 2.34, 8), sweeps=40000)
    cr = fss.crossings(res)[0]
    tc = 2.0 / math.log(1.0 + math.sqrt(2.0))
    assert cr["T_cross"] is not None
    assert abs(cr["T_cross"] - tc) < max(0.02, 5 * (cr["err"] or 0.0))
