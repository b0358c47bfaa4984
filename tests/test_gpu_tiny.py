"""GPU parity of the one-CTA kernel (the whole lattice in shared memory, every
sweep of a call in one launch; launch configurations with proc_bits == 8),
against the oracle, bit for bit.

It is the default for L <= 512, so the other parity tests at those sizes run
through it too; here every block size and every size it takes (64 .. 1024, up
to 128 KiB of shared memory and 256 bytes per thread) is checked, with samples
recorded every sweep, every third sweep across split calls, and not at all.
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


TINY = {"proc_bits": 8, "regcap": 0, "insert": 0, "grid": 1, "persistent": 0}


@pytest.mark.parametrize("L", [64, 128, 256, 512, 1024])
@pytest.mark.parametrize("block", [128, 256, 512])
@pytest.mark.parametrize("tpw", [1, 2, 4])
def test_tiny_sizes_blocks_and_threads_per_word_bit_exact(P, orc, L, block, tpw):
    n = 12 if L <= 256 else 3
    T, seed, sid = TC, L + block + tpw, 1
    lat = P.Lattice(L, T, seed=seed, stream_id=sid, init="hot", word_bits=64 if L >= 512 else 32)
    lat.set_launch(**TINY, block=block, rows_per_item=tpw)
    assert lat.launch["proc_bits"] == 8
    M, E = lat.sweep(n, 1, collect=True)
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_hot(L, seed, sid)
    Mo, Eo = orc.run(s, n, seed, sid, thr4, thr8)
    assert np.array_equal(M, Mo) and np.array_equal(E, Eo)
    assert np.array_equal(lat.spins(), s)
    assert lat.recount() == orc.recount(s)
    lat.close()


@pytest.mark.parametrize("T", [0.8, 2.0, 3.5])
def test_tiny_split_calls_sparse_records_and_final_state(P, orc, T):
    """record_every = 3 over calls of 7, 13, 1, 39 and 2 sweeps (the sample phase
    crosses call boundaries); calls with no sample still update M and E."""
    L, seed = 128, 41
    lat = P.Lattice(L, T, seed=seed, init="cold_up")
    lat.set_launch(**TINY, block=256, rows_per_item=2)
    Ms, Es = [], []
    for n in (7, 13, 1, 39, 2):
        M, E = lat.sweep(n, 3, collect=True)
        Ms.append(M)
        Es.append(E)
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_cold(L, 1)
    Mo, Eo = orc.run(s, 62, seed, 0, thr4, thr8)
    assert np.array_equal(np.concatenate(Ms), Mo[2::3]) and np.array_equal(np.concatenate(Es), Eo[2::3])
    d = lat.measure()
    assert (d["M"], d["E"]) == (int(Mo[-1]), int(Eo[-1]))
    lat.sweep(5, 0)  # nothing recorded, the final state is still counted
    Mo2, Eo2 = orc.run(s, 5, seed, 0, thr4, thr8, t0=62)
    d = lat.measure()
    assert (d["M"], d["E"]) == (int(Mo2[-1]), int(Eo2[-1]))
    assert np.array_equal(lat.spins(), s)


def test_tiny_equals_plain_launches_on_the_L64_workload(P):
    """L = 64, cold start, 1000 sweeps, M/E every sweep: one launch of the one-CTA
    kernel and 2000 launches of the step kernel give the same lattice and samples."""
    a = P.Lattice(64, TC, seed=1, init="cold_up")
    assert a.launch["proc_bits"] == 8  # the default at this size
    b = P.Lattice(64, TC, seed=1, init="cold_up")
    b.set_launch(proc_bits=32, regcap=0, insert=0, block=128, rows_per_item=4, grid=0)
    Ma, Ea = a.sweep(1000, 1, collect=True)
    Mb, Eb = b.sweep(1000, 1, collect=True)
    assert np.array_equal(Ma, Mb) and np.array_equal(Ea, Eb)
    assert np.array_equal(a.spins(), b.spins())


def test_tiny_is_rejected_where_it_does_not_apply(P):
    for L in (192, 2048):
        lat = P.Lattice(L, 2.0, seed=1)
        with pytest.raises(P.IsingError):
            lat.set_launch(**TINY, block=256, rows_per_item=1)
        lat.close()
    lat = P.Lattice(128, 2.0, seed=1)
    with pytest.raises(P.IsingError):
        lat.set_launch(**TINY, block=1024, rows_per_item=1)
    lat.close()
    lat = P.Lattice(64, 2.0, seed=1)
    # 1024 threads is the warp-specialised form: L = 64 or 128, one thread per
    # word, one CTA (L = 64 only) or a cluster of 2, 4 or 8
    for bad in ({"block": 1024, "rows_per_item": 2}, {"block": 1024, "grid": 3}, {"block": 1024, "grid": 16},
                {"grid": 3}, {"grid": 16}, {"rows_per_item": 3}, {"rows_per_item": 8}, {"regcap": 1}):
        cfg = dict(TINY, block=256, rows_per_item=1)
        cfg.update(bad)
        with pytest.raises(P.IsingError):
            lat.set_launch(**cfg)
    lat.close()


def test_tiny_autotune_and_strips_keep_step_kernels(P, orc):
    """The autotuner may pick the one-CTA kernel for a small lattice; the strip and
    allocation-free entry points, which run single steps, still use step kernels."""
    L, T, seed = 128, TC, 3
    lat = P.Lattice(L, T, seed=seed)
    cfg, us = lat.autotune(reps=1)
    assert cfg in P.ising_launch_candidates(L) and us > 0
    M, E = lat.sweep(6, 1, collect=True)
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_hot(L, seed)
    Mo, Eo = orc.run(s, 6, seed, 0, thr4, thr8)
    assert np.array_equal(M, Mo) and np.array_equal(E, Eo)


@pytest.mark.parametrize("L", [64, 256, 1024])
@pytest.mark.parametrize("H", [0.3, -2.0, 5.0])
def test_tiny_in_a_field_bit_exact(P, orc, L, H):
    """The one-CTA kernel in a field (ten classes, one thread per word whatever the
    configuration's threads per word) against the oracle's field update."""
    n = 10 if L <= 256 else 3
    T, seed = 2.1, L + 17
    lat = P.Lattice(L, T, seed=seed, init="hot", H=H)
    lat.set_launch(**TINY, block=256, rows_per_item=4)
    M, E = lat.sweep(n, 1, collect=True)
    s = orc.init_hot(L, seed, 0)
    Mo, Eo = orc.run_field(s, n, seed, 0, T, H)
    assert np.array_equal(M, Mo) and np.array_equal(E, Eo)
    assert np.array_equal(lat.spins(), s)
    # a change of the field between calls keeps the one-CTA path
    lat.set_field(-H)
    M2, _ = lat.sweep(4, 2, collect=True)
    Mo2, _ = orc.run_field(s, 4, seed, 0, T, -H, t0=n)
    recorded = [i for i in range(4) if (n + i + 1) % 2 == 0]  # sweep t is recorded when (t + 1) % 2 == 0
    assert np.array_equal(M2, Mo2[recorded])
    assert np.array_equal(lat.spins(), s)


@pytest.mark.parametrize("L", [64, 128, 256, 1024])
@pytest.mark.parametrize("ctas", [2, 4, 8])
@pytest.mark.parametrize("tpw", [1, 4])
def test_tiny_cluster_bit_exact(P, orc, L, ctas, tpw):
    """A thread-block cluster of 2, 4 or 8 CTAs sharing one lattice (each holds
    L / ctas rows and reads its halo rows from its neighbours' shared memory)."""
    n = 10 if L <= 256 else 3
    T, seed, sid = 2.2, L + ctas + tpw, 3
    lat = P.Lattice(L, T, seed=seed, stream_id=sid, init="hot")
    lat.set_launch(**dict(TINY, grid=ctas), block=256, rows_per_item=tpw)
    M, E = lat.sweep(n, 1, collect=True)
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_hot(L, seed, sid)
    Mo, Eo = orc.run(s, n, seed, sid, thr4, thr8)
    assert np.array_equal(M, Mo) and np.array_equal(E, Eo)
    assert np.array_equal(lat.spins(), s)
    # sparse records over split calls, then a field
    M2, _ = lat.sweep(7, 3, collect=True)
    Mo2, _ = orc.run(s, 7, seed, sid, thr4, thr8, t0=n)
    assert np.array_equal(M2, Mo2[[i for i in range(7) if (n + i + 1) % 3 == 0]])
    lat.set_field(0.7)
    M3, E3 = lat.sweep(4, 1, collect=True)
    Mo3, Eo3 = orc.run_field(s, 4, seed, sid, T, 0.7, t0=n + 7)
    assert np.array_equal(M3, Mo3) and np.array_equal(E3, Eo3)
    assert np.array_equal(lat.spins(), s)
    lat.close()


WS_SHAPES = [(64, 1), (64, 2), (64, 4), (64, 8), (128, 2), (128, 4), (128, 8), (256, 2), (256, 4), (256, 8)]


@pytest.mark.parametrize("L,ctas", WS_SHAPES)
def test_warp_specialised_is_bit_exact(P, orc, L, ctas):
    """1024 threads and one thread per word run the warp-specialised kernel
    (producer warps draw the masks into a ring, consumer warps update; with a
    cluster the producers sit in the other CTAs and store into the first CTA's
    ring through distributed shared memory): lattice and every sample against
    the oracle, for several call splits and sample spacings, both parities of
    the start sweep and record_every = 0."""
    T, seed, sid = 2.269185, 17, 5
    thr4, thr8 = orc.thresholds(T)
    lat = P.Lattice(L, T, seed=seed, stream_id=sid, init="hot")
    lat.set_launch(proc_bits=8, regcap=0, insert=0, block=1024, rows_per_item=1, grid=ctas, persistent=0)
    s = orc.init_hot(L, seed, sid)
    t = 0
    for n, rec in ((1, 1), (7, 3), (300, 1), (129, 64), (5, 0), (1000, 7)):
        got = lat.sweep(n, rec, collect=bool(rec))
        Mo, Eo = orc.run(s, n, seed, sid, thr4, thr8, t0=t)
        if rec:
            k0 = (rec - 1 - t) % rec  # first recorded sweep of this call
            assert np.array_equal(got[0], Mo[k0::rec]) and np.array_equal(got[1], Eo[k0::rec]), (n, rec)
        assert (lat.measure()["M"], lat.measure()["E"]) == (Mo[-1], Eo[-1])
        t += n
    assert np.array_equal(lat.spins(), s)
    lat.close()


@pytest.mark.parametrize("L,ctas,hold", [(64, 1, 6), (64, 4, 6), (128, 8, 6), (256, 8, 6), (64, 1, 20), (64, 4, 20),
                                         (128, 8, 20), (256, 8, 20)])
def test_warp_specialised_wait_runs_out_and_reports(P, monkeypatch, L, ctas, hold):
    """A step whose masks are never announced (a middle step, or the last of
    the call's 20): the consumers' bounded wait runs out, the call reports
    ISING_ERR_TIMEOUT, the handle is failed, and the GPU stays usable."""
    lat = P.Lattice(L, 2.0, seed=1, init="hot")
    lat.set_launch(proc_bits=8, regcap=0, insert=0, block=1024, rows_per_item=1, grid=ctas, persistent=0)
    monkeypatch.setenv("ISING_TINY_HOLD_STEP", str(hold))
    with pytest.raises(P.IsingError) as ei:
        lat.sweep(10, 1, collect=True)
    assert ei.value.status == P.ERR_TIMEOUT
    monkeypatch.delenv("ISING_TINY_HOLD_STEP")
    with pytest.raises(P.IsingError) as ei:
        lat.sweep(1, 1)
    assert ei.value.status == P.ERR_STATE
    lat.close()
    ok = P.Lattice(L, 2.0, seed=1, init="hot")
    ok.sweep(10, 1)
    assert ok.measure()["sweeps_done"] == 10
    ok.close()


@pytest.mark.parametrize("L,ctas", [(64, 1), (128, 4), (256, 8)])
def test_warp_specialised_configuration_in_a_field_runs_the_field_kernel(P, orc, L, ctas):
    """The warp-specialised configuration has no field form: in a field the
    one-CTA or cluster field kernel runs instead, bit-exact with the oracle."""
    T, H, seed = 2.1, 0.3, 9
    lat = P.Lattice(L, T, seed=seed, init="hot", H=H)
    lat.set_launch(proc_bits=8, regcap=0, insert=0, block=1024, rows_per_item=1, grid=ctas, persistent=0)
    M, E = lat.sweep(12, 1, collect=True)
    s = orc.init_hot(L, seed, 0)
    Mo, Eo = orc.run_field(s, 12, seed, 0, T, H)
    assert np.array_equal(M, Mo) and np.array_equal(E, Eo)
    assert np.array_equal(lat.spins(), s)
    lat.close()


@pytest.mark.parametrize("L,launch", [(64, None), (128, None), (256, None), (512, None),
                                      (64, dict(TINY, block=1024, rows_per_item=1, grid=1)),
                                      (128, dict(TINY, block=256, rows_per_item=2))])
def test_long_calls_run_as_several_launches(P, orc, monkeypatch, L, launch):
    """A call longer than one launch's sweep bound runs as several launches
    (forced here with a bound of 7 sweeps): the lattice and every sample equal
    the oracle's, with samples spread over the launches and a final state slot
    that each launch hands to the next."""
    T, seed, sid = 2.269185, 23, 2
    thr4, thr8 = orc.thresholds(T)
    lat = P.Lattice(L, T, seed=seed, stream_id=sid, init="hot")
    if launch is not None:
        lat.set_launch(**launch)
    monkeypatch.setenv("ISING_TINY_MAX_SWEEPS", "7")
    s = orc.init_hot(L, seed, sid)
    t = 0
    for n, rec in ((50, 3), (15, 0), (22, 1)):
        got = lat.sweep(n, rec, collect=bool(rec))
        Mo, Eo = orc.run(s, n, seed, sid, thr4, thr8, t0=t)
        if rec:
            k0 = (rec - 1 - t) % rec
            assert np.array_equal(got[0], Mo[k0::rec]) and np.array_equal(got[1], Eo[k0::rec]), (n, rec)
        d = lat.measure()
        assert (d["M"], d["E"]) == (Mo[-1], Eo[-1])
        t += n
    assert np.array_equal(lat.spins(), s)
    lat.close()


def test_long_calls_in_a_field_run_as_several_launches(P, orc, monkeypatch):
    L, T, H, seed = 64, 2.1, 0.3, 9
    lat = P.Lattice(L, T, seed=seed, init="hot", H=H)
    monkeypatch.setenv("ISING_TINY_MAX_SWEEPS", "5")
    M, E = lat.sweep(23, 2, collect=True)
    s = orc.init_hot(L, seed, 0)
    Mo, Eo = orc.run_field(s, 23, seed, 0, T, H)
    assert np.array_equal(M, Mo[1::2]) and np.array_equal(E, Eo[1::2])
    assert np.array_equal(lat.spins(), s)
    lat.close()
