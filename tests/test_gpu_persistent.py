"""GPU parity of the persistent form (launch configurations with persistent = 1:
every sweep of an ising_sweep call in one cooperative launch, a grid-wide barrier
between the checkerboard steps) against the oracle, bit for bit: both word
widths, every register cap, ragged lattices, and call splits where the call's
last sweep is recorded, is not, or nothing is recorded."""
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


@pytest.mark.parametrize("L", [64, 192, 1088, 2048])
@pytest.mark.parametrize("proc_bits,regcap,block,R", [(32, 0, 256, 2), (64, 1, 512, 8), (64, 2, 256, 4),
                                                       (32, 2, 512, 8), (64, 0, 512, 2)])
def test_persistent_shapes_bit_exact(P, orc, L, proc_bits, regcap, block, R):
    if L % R or L % proc_bits:
        pytest.skip("shape not valid for this L")
    T, seed, sid = TC, L + block + R, 2
    lat = P.Lattice(L, T, seed=seed, stream_id=sid, init="hot", word_bits=32 if proc_bits == 32 else 64)
    lat.set_launch(proc_bits=proc_bits, regcap=regcap, insert=0, block=block, rows_per_item=R, grid=0,
                   persistent=1)
    assert lat.launch["persistent"] == 1
    n = 9 if L <= 1088 else 4
    M, E = lat.sweep(n, 1, collect=True)
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_hot(L, seed, sid)
    Mo, Eo = orc.run(s, n, seed, sid, thr4, thr8)
    assert np.array_equal(M, Mo) and np.array_equal(E, Eo)
    assert np.array_equal(lat.spins(), s)
    lat.close()


def test_persistent_split_calls_and_final_state(P, orc):
    """record_every = 3 over calls of 7, 13, 1, 39 and 2 sweeps; calls whose last
    sweep is recorded write it to both slots; calls with nothing recorded still
    update M and E; a field change between calls runs the field kernel."""
    L, T, seed = 320, 2.1, 17
    lat = P.Lattice(L, T, seed=seed, init="cold_up")
    lat.set_launch(proc_bits=64, regcap=2, insert=0, block=256, rows_per_item=4, grid=0, persistent=1)
    Ms = []
    for n in (7, 13, 1, 39, 2):
        M, _ = lat.sweep(n, 3, collect=True)
        Ms.append(M)
        d = lat.measure()
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_cold(L, 1)
    Mo, Eo = orc.run(s, 62, seed, 0, thr4, thr8)
    assert np.array_equal(np.concatenate(Ms), Mo[2::3])
    assert (d["M"], d["E"]) == (int(Mo[-1]), int(Eo[-1]))
    lat.sweep(4, 0)
    Mo2, Eo2 = orc.run(s, 4, seed, 0, thr4, thr8, t0=62)
    d = lat.measure()
    assert (d["M"], d["E"]) == (int(Mo2[-1]), int(Eo2[-1]))
    lat.set_field(0.4)
    M3, _ = lat.sweep(5, 1, collect=True)
    Mo3, _ = orc.run_field(s, 5, seed, 0, T, 0.4, t0=66)
    assert np.array_equal(M3, Mo3)
    assert np.array_equal(lat.spins(), s)
    lat.close()


def test_persistent_is_rejected_where_it_does_not_apply(P):
    lat = P.Lattice(256, 2.0, seed=1)
    base = dict(proc_bits=32, regcap=0, insert=0, block=256, rows_per_item=4, grid=0, persistent=1)
    for bad in ({"insert": 1}, {"regcap": 3}, {"grid": 8}, {"proc_bits": 8}):
        cfg = dict(base)
        cfg.update(bad)
        with pytest.raises(P.IsingError):
            lat.set_launch(**cfg)
    lat.set_launch(**base)
    lat.close()
