"""ising_sweep_noalloc: the sweep for callers that cannot allocate memory.

Callers that own all of their device memory (a pool that has reserved the HBM
budget, a host application lending buffers to a plug-in) use this entry point:
it runs the sweep on the caller's lattice and keeps its scratch in a fixed
array inside the library.  Its results must equal those of ising_sweep.  This
file is collected last so that a run stopping at the first failure has already
run every other test; it passes alone in a fresh process too (the first call
performs the per-device set-up).
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


@pytest.mark.parametrize("L,word_bits,record_every", [(64, 32, 1), (256, 32, 1), (1024, 64, 3), (4096, 32, 2)])
def test_noalloc_matches_ising_sweep_on_two_calls(P, L, word_bits, record_every):
    import torch

    T, seed, stream_id = 2.269185, 31, 6
    ref = P.Lattice(L, T, seed=seed, stream_id=stream_id, init="hot", word_bits=word_bits)
    # the caller's own device lattice, a copy of the same hot start
    packed = ref.packed()
    dev = torch.from_numpy(packed.view(np.int64).copy()).cuda()
    torch.cuda.synchronize()
    t0 = 0
    for n in (40, 25):  # two calls in a row
        k = (t0 + n) // record_every - t0 // record_every
        Mr, Er = ref.sweep(n, record_every, collect=True)
        M = np.zeros(k, dtype=np.int64)
        E = np.zeros(k, dtype=np.int64)
        P.ising_sweep_noalloc(dev.data_ptr(), L, word_bits, T, seed, stream_id, t0, n,
                              record_every, M, E, k)
        assert np.array_equal(M, Mr) and np.array_equal(E, Er)
        got = dev.cpu().numpy().view(packed.dtype).reshape(packed.shape)
        assert np.array_equal(got, ref.packed())
        t0 += n
    ref.close()


@pytest.mark.parametrize("L", [64, 256, 512])
def test_noalloc_long_calls_run_as_several_launches(P, monkeypatch, L):
    """The small-lattice kernels take at most 2^30 sweeps per launch (forced
    down to 6 here): the samples spread over the launches and the state after
    the call equal ising_sweep's."""
    import torch

    T, seed, stream_id = 2.269185, 41, 3
    ref = P.Lattice(L, T, seed=seed, stream_id=stream_id, init="hot", word_bits=32)
    packed = ref.packed()
    dev = torch.from_numpy(packed.view(np.int64).copy()).cuda()
    torch.cuda.synchronize()
    Mr, Er = ref.sweep(40, 3, collect=True)
    k = 40 // 3
    M = np.zeros(k, dtype=np.int64)
    E = np.zeros(k, dtype=np.int64)
    monkeypatch.setenv("ISING_TINY_MAX_SWEEPS", "6")
    P.ising_sweep_noalloc(dev.data_ptr(), L, 32, T, seed, stream_id, 0, 40, 3, M, E, k)
    assert np.array_equal(M, Mr) and np.array_equal(E, Er)
    got = dev.cpu().numpy().view(packed.dtype).reshape(packed.shape)
    assert np.array_equal(got, ref.packed())
    ref.close()


def test_noalloc_rejects_more_samples_than_its_scratch(P):
    import torch

    L = 64
    dev = torch.zeros(L * L // 8, dtype=torch.uint8, device="cuda")
    cap = 70000
    M = np.zeros(cap, dtype=np.int64)
    E = np.zeros(cap, dtype=np.int64)
    with pytest.raises(P.IsingError) as ei:
        P.ising_sweep_noalloc(dev.data_ptr(), L, 32, 2.0, 1, 0, 0, 65537, 1, M, E, cap)
    assert ei.value.status == P.ERR_INVALID and "split" in P.ising_last_error()
    # nothing ran: the lattice is untouched
    assert int(dev.sum().item()) == 0


def test_noalloc_fills_its_whole_scratch(P):
    """Exactly ISING_NOALLOC_MAX_RECORDS samples in one call (every slot of the
    fixed array) on L = 64, against ising_sweep."""
    import torch

    L, T, seed, n = 64, 2.269185, 5, 65536
    ref = P.Lattice(L, T, seed=seed, init="hot")
    packed = ref.packed()
    dev = torch.from_numpy(packed.view(np.int64).copy()).cuda()
    Mr, Er = ref.sweep(n, 1, collect=True)
    M = np.zeros(n, dtype=np.int64)
    E = np.zeros(n, dtype=np.int64)
    P.ising_sweep_noalloc(dev.data_ptr(), L, 32, T, seed, 0, 0, n, 1, M, E, n)
    assert np.array_equal(M, Mr) and np.array_equal(E, Er)
    got = dev.cpu().numpy().view(packed.dtype).reshape(packed.shape)
    assert np.array_equal(got, ref.packed())
    ref.close()


@pytest.mark.parametrize("L", [64, 2048])
def test_noalloc_without_samples(P, L):
    """record_every = 0: no sample, the call returns once the work is queued."""
    import torch

    T, seed = 2.0, 8
    ref = P.Lattice(L, T, seed=seed, init="hot")
    packed = ref.packed()
    dev = torch.from_numpy(packed.view(np.int64).copy()).cuda()
    ref.sweep(30, 0)
    P.ising_sweep_noalloc(dev.data_ptr(), L, 32, T, seed, 0, 0, 30, 0)
    torch.cuda.synchronize()
    got = dev.cpu().numpy().view(packed.dtype).reshape(packed.shape)
    assert np.array_equal(got, ref.packed())
    ref.close()


def test_noalloc_rejects_misaligned_and_host_lattices(P):
    import torch

    L = 64
    dev = torch.zeros(L * L // 8 + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.IsingError) as ei:
        P.ising_sweep_noalloc(dev.data_ptr() + 4, L, 32, 2.0, 1, 0, 0, 10, 0)
    assert ei.value.status == P.ERR_INVALID and "aligned" in P.ising_last_error()
    torch.cuda.synchronize()
    assert int(dev.sum().item()) == 0
    # a host array is refused; with zero sweeps nothing would be launched even
    # if it were not
    host = np.zeros(L * L // 8 + 64, dtype=np.uint8)
    addr = host.ctypes.data + (-host.ctypes.data) % 16
    with pytest.raises(P.IsingError) as ei:
        P.ising_sweep_noalloc(addr, L, 32, 2.0, 1, 0, 0, 0, 0)
    assert ei.value.status == P.ERR_INVALID and "device memory" in P.ising_last_error()
    # the sweep counter guard does not wrap around
    with pytest.raises(P.IsingError):
        P.ising_sweep_noalloc(dev.data_ptr(), L, 32, 2.0, 1, 0, 2 ** 64 - 1, 2, 0)
    # the binding refuses sample arrays of the wrong type or size
    with pytest.raises(ValueError):
        P.ising_sweep_noalloc(dev.data_ptr(), L, 32, 2.0, 1, 0, 0, 4, 1, np.zeros(4), np.zeros(4), 4)
    with pytest.raises(ValueError):
        P.ising_sweep_noalloc(dev.data_ptr(), L, 32, 2.0, 1, 0, 0, 4, 1, np.zeros(3, np.int64),
                              np.zeros(3, np.int64), 4)
