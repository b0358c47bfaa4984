"""Randomised parity: whole configurations drawn from a seeded generator, each run
through the C ABI and compared with the oracle bit for bit.

A case draws L (a multiple of 64 up to 512), T, a field H (zero half of the
time), the initial state (hot, cold +1 / -1, a random int8 buffer), the storage
word width, any launch configuration the library lists for that L (the one-CTA
form included), how the sweeps are split over calls, the sample spacing, and
temperature / field changes between calls.  Batch cases put several such
lattices into one persistent launch instead.  Every recorded M and E and the
final lattice must equal the oracle's.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1007_3726_gb300 as P

    P.build()
    P.load()
    return P


def _draw(rng):
    L = int(rng.choice([64, 128, 192, 256, 320, 384, 448, 512]))
    init = str(rng.choice(["hot", "cold_up", "cold_down", "buffer"]))
    c = dict(L=L, T=float(rng.uniform(0.5, 5.0)), H=float(rng.uniform(-3, 3)) if rng.random() < 0.5 else 0.0,
             seed=int(rng.integers(0, 2 ** 63)), stream_id=int(rng.integers(0, 1000)), init=init,
             word_bits=int(rng.choice([0, 32, 64])), record_every=int(rng.choice([0, 1, 2, 3, 5])))
    if init == "buffer":
        c["buf"] = np.where(rng.random((L, L)) < rng.uniform(0.1, 0.9), 1, -1).astype(np.int8)
    # calls: (sweeps, T, H) with the parameters changed before some calls
    calls, T, H = [], c["T"], c["H"]
    for _ in range(int(rng.integers(1, 4))):
        if rng.random() < 0.3:
            T = float(rng.uniform(0.5, 5.0))
        if rng.random() < 0.3:
            H = float(rng.uniform(-3, 3)) if rng.random() < 0.5 else 0.0
        calls.append((int(rng.integers(1, 8)), T, H))
    c["calls"] = calls
    return c


def _start(orc, c):
    L = c["L"]
    if c["init"] == "hot":
        return orc.init_hot(L, c["seed"], c["stream_id"])
    if c["init"] == "cold_up":
        return orc.init_cold(L, 1)
    if c["init"] == "cold_down":
        return orc.init_cold(L, -1)
    return np.ascontiguousarray(c["buf"])


def _oracle(orc, c):
    """Samples of every call and the final lattice from the oracle."""
    s = _start(orc, c)
    t, out = 0, []
    for n, T, H in c["calls"]:
        if H == 0.0:
            thr4, thr8 = orc.thresholds(T)
            M, E = orc.run(s, n, c["seed"], c["stream_id"], thr4, thr8, t0=t)
        else:
            M, E = orc.run_field(s, n, c["seed"], c["stream_id"], T, H, t0=t)
        re = c["record_every"]
        sel = [i for i in range(n) if re and (t + i + 1) % re == 0]
        out.append((M[sel], E[sel]))
        t += n
    return out, s


def _lattice(P, c):
    return P.Lattice(c["L"], c["T"], seed=c["seed"], stream_id=c["stream_id"], init=c["init"],
                     spins=c.get("buf"), word_bits=c["word_bits"], H=c["H"])


@pytest.mark.parametrize("case", range(48))
def test_random_configuration_bit_exact(P, orc, case):
    rng = np.random.default_rng(1000 + case)
    c = _draw(rng)
    lat = _lattice(P, c)
    cands = P.ising_launch_candidates(c["L"])
    cfg = cands[int(rng.integers(0, len(cands)))]
    lat.set_launch(**cfg)
    want, s = _oracle(orc, c)
    for (n, T, H), (Mo, Eo) in zip(c["calls"], want):
        lat.set_temperature(T)
        lat.set_field(H)
        if c["record_every"]:
            M, E = lat.sweep(n, c["record_every"], collect=True)
            assert np.array_equal(M, Mo) and np.array_equal(E, Eo), (c["L"], cfg, n, T, H)
        else:
            lat.sweep(n, 0)
    assert np.array_equal(lat.spins(), s), (c["L"], cfg)
    assert lat.recount() == orc.recount(s)
    lat.close()


@pytest.mark.parametrize("case", range(8))
def test_random_batch_bit_exact(P, orc, case):
    """Several random lattices (one call each, fixed T and H) in one persistent launch."""
    rng = np.random.default_rng(5000 + case)
    cs = []
    for _ in range(int(rng.integers(2, 7))):
        c = _draw(rng)
        c["calls"] = [(int(rng.integers(1, 9)), c["T"], c["H"])]
        c["record_every"] = int(rng.choice([1, 2, 3]))
        cs.append(c)
    lats = [_lattice(P, c) for c in cs]
    re = [c["record_every"] for c in cs]
    # one batch records with one spacing: use the first lattice's for all
    with P.Batch(lats, [c["calls"][0][0] for c in cs], re[0]) as b:
        b.run(1)
    for c, lat in zip(cs, lats):
        c["record_every"] = re[0]
        [(Mo, Eo)], s = _oracle(orc, c)
        M, E = lat.samples()
        assert np.array_equal(M, Mo) and np.array_equal(E, Eo), (c["L"], c["H"])
        assert np.array_equal(lat.spins(), s), (c["L"], c["H"])
        lat.close()
