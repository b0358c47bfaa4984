"""Row strips on the GPU with emulated ranks (one process, halo rows copied
between the strips before every step): the production strip kernel for 1-5
ranks and uneven splits must equal the one-lattice path bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1007_3726_gb300 as P

    P.build()
    P.load()
    return P


@pytest.mark.parametrize("world,L,wb", [(1, 256, 64), (2, 256, 32), (3, 320, 64), (5, 1024, 32),
                                        (4, 2048, 64)])
def test_emulated_ranks_equal_one_lattice(P, world, L, wb):
    import torch

    from paper_1007_3726_gb300.distributed import LocalExchange, StripLattice, sweep_strips

    T, seed, sid, n, rec = 2.269185, 17, 3, 7, 1
    strips = [StripLattice(L, T, seed=seed, stream_id=sid, init="hot", rank=k, world=world, word_bits=wb)
              for k in range(world)]
    M, E = sweep_strips(strips, LocalExchange(), L, n, rec)
    ref = P.Lattice(L, T, seed=seed, stream_id=sid, init="hot", word_bits=wb)
    Mr, Er = ref.sweep(n, rec, collect=True)
    assert M == [int(v) for v in Mr] and E == [int(v) for v in Er]
    full = torch.cat([s.rows() for s in strips]).cpu().numpy()
    assert full.tobytes() == ref.packed().tobytes()


def test_strip_cold_start_and_errors(P):
    import torch

    from paper_1007_3726_gb300.distributed import LocalExchange, StripLattice, sweep_strips

    strips = [StripLattice(128, 0.01, init="cold_up", rank=k, world=2) for k in range(2)]
    M, E = sweep_strips(strips, LocalExchange(), 128, 3, 1)
    assert M == [128 * 128] * 3 and E == [-2 * 128 * 128] * 3
    buf = torch.zeros((4, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(P.IsingError):
        P.ising_strip_step(buf.data_ptr(), 128, 64, 127, 2, 2.0, 1, 0, 0, 0)   # rows beyond L
    with pytest.raises(P.IsingError):
        P.ising_strip_step(buf.data_ptr(), 128, 64, 0, 2, 2.0, 1, 0, 0, 2)     # p out of range


@pytest.mark.parametrize("world,L,wb", [(3, 320, 64), (3, 448, 32)])
def test_three_gpu_strips_equal_the_oracle(P, orc, world, L, wb):
    """Three strips of uneven height (emulated ranks on one GPU, halo rows copied
    between them before every step): the whole lattice and every M/E sample
    against the oracle run of the same lattice."""
    import torch

    from paper_1007_3726_gb300.distributed import LocalExchange, StripLattice, sweep_strips

    T, seed, sid, n = 2.3, 41, 9, 6
    strips = [StripLattice(L, T, seed=seed, stream_id=sid, init="hot", rank=k, world=world, word_bits=wb)
              for k in range(world)]
    M, E = sweep_strips(strips, LocalExchange(), L, n, 1)
    thr4, thr8 = orc.thresholds(T)
    s = orc.init_hot(L, seed, sid)
    Mo, Eo = orc.run(s, n, seed, sid, thr4, thr8)
    assert M == [int(v) for v in Mo] and E == [int(v) for v in Eo]
    packed = torch.cat([st.rows() for st in strips]).cpu().numpy().view(np.uint8).reshape(L, L // 8)
    spins = np.unpackbits(packed, axis=1, bitorder="little").astype(np.int8) * 2 - 1
    assert np.array_equal(spins, s)
