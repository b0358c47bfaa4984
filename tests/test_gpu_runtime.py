"""Runtime pieces around the sweep: checkpoint / resume, the allocator hook
(PyTorch's caching allocator, and an injected allocation failure), handle
errors."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1007_3726_gb300 as P

    P.build()
    P.load()
    return P


@pytest.mark.parametrize("word_bits", [32, 64])
def test_checkpoint_resume_is_bit_exact(P, tmp_path, word_bits):
    L, T = 512, 2.269185
    ref = P.Lattice(L, T, seed=21, stream_id=4, init="hot", word_bits=word_bits)
    Ma, Ea = ref.sweep(10, 2, collect=True)
    path = str(tmp_path / "ckpt.npz")
    ref.save(path)
    Mb, Eb = ref.sweep(15, 2, collect=True)
    res = P.Lattice.load(path)
    assert res.sweeps_done == 10
    M0, E0 = res.restored_samples
    assert np.array_equal(M0, Ma) and np.array_equal(E0, Ea)
    Mc, Ec = res.sweep(15, 2, collect=True)
    assert np.array_equal(Mb, Mc) and np.array_equal(Eb, Ec)
    assert np.array_equal(ref.spins(), res.spins())
    assert res.measure()["sweeps_done"] == 25


def test_torch_caching_allocator_hook(P):
    import torch

    P.use_torch_allocator()
    try:
        a = P.Lattice(256, 2.0, seed=3, init="hot")
        Ma, Ea = a.sweep(12, 1, collect=True)
        sa = a.spins()
        a.close()
    finally:
        P.ising_set_allocator(None)
    b = P.Lattice(256, 2.0, seed=3, init="hot")
    Mb, Eb = b.sweep(12, 1, collect=True)
    assert np.array_equal(Ma, Mb) and np.array_equal(Ea, Eb) and np.array_equal(sa, b.spins())
    torch.cuda.synchronize()


def test_injected_allocation_failure(P):
    """An allocator that fails: creation reports ISING_ERR_OOM, frees what it took,
    and the library keeps working once a working allocator is back."""
    import torch

    taken = {}

    def alloc(n, s):
        if n > 4096:  # the lattice and staging buffers fail, small ones succeed
            return None
        p = torch.cuda.caching_allocator_alloc(n)
        taken[p] = n
        return p

    def release(p, s):
        taken.pop(p, None)
        torch.cuda.caching_allocator_delete(p)

    P.ising_set_allocator(alloc, release)
    try:
        with pytest.raises(P.IsingError) as ei:
            P.Lattice(1024, 2.0, seed=1)
        assert ei.value.status == P.ERR_OOM
        assert not taken  # nothing left allocated
    finally:
        P.ising_set_allocator(None)
    ok = P.Lattice(1024, 2.0, seed=1)
    ok.sweep(2)
    assert ok.measure()["sweeps_done"] == 2


def test_invalid_first_sweep_and_counter_limit(P):
    with pytest.raises(P.IsingError):
        P.Lattice(256, 2.0, first_sweep=2 ** 32 - 1)
    lat = P.Lattice(256, 2.0, first_sweep=2 ** 32 - 3)
    lat.sweep(1)
    with pytest.raises(P.IsingError) as ei:
        lat.sweep(1)
    assert ei.value.status == P.ERR_INVALID
