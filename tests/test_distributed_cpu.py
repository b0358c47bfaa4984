"""The row-strip decomposition's exchange over real torch.distributed ranks
(gloo, world sizes 2 and 3, CPU): each rank holds a strip with halo rows, the
ranks swap boundary rows before every checkerboard step and sum their counts at
recorded sweeps.  The strip's own update is the oracle's window step here (no
GPU), so the test checks the exchange protocol and the count reduction: the
assembled lattice and every (M, E) sample must equal the oracle's whole-lattice
run."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1007_3726_gb300.distributed import TorchDistExchange, strip_rows, sweep_strips


class OracleStrip:
    """A strip of int8 spins with halo rows, updated by the oracle's window step."""

    def __init__(self, orc, L, T, seed, sid, rank, world):
        self.orc, self.L, self.seed, self.sid = orc, L, seed, sid
        self.thr4, self.thr8 = orc.thresholds(T)
        self.r0, self.n = strip_rows(L, rank, world)
        self.buf = np.zeros((self.n + 2, L), dtype=np.int8)
        self.buf[1:self.n + 1] = orc.init_hot(L, seed, sid, row0=self.r0, nrows=self.n)
        self.t = 0
        self._c = torch.zeros(2, dtype=torch.int64)

    def boundary_rows(self):
        return torch.from_numpy(self.buf[1].copy()), torch.from_numpy(self.buf[self.n].copy())

    def set_halos(self, top, bottom):
        self.buf[0] = top.numpy()
        self.buf[self.n + 1] = bottom.numpy()

    def step(self, p, count=False):
        self.orc.half_sweep(self.buf, t=self.t, p=p, seed=self.seed, stream_id=self.sid, thr4=self.thr4,
                            thr8=self.thr8, L=self.L, row0=(self.r0 - 1) % self.L, periodic=False)
        if count:
            s = self.buf.astype(np.int64)
            rows = s[1:self.n + 1]
            y = np.arange(self.r0, self.r0 + self.n)[:, None]
            x = np.arange(self.L)[None, :]
            odd = ((x + y) & 1) == 1
            nb = [s[0:self.n], s[2:self.n + 2], np.roll(rows, 1, 1), np.roll(rows, -1, 1)]
            anti = sum(int(((rows != v) & odd).sum()) for v in nb)
            self._c += torch.tensor([int((rows == 1).sum()), anti], dtype=torch.int64)

    def zero_counts(self):
        self._c.zero_()

    def counts(self):
        return self._c


def _worker(rank, world, port, L, T, n, rec, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle

        strip = OracleStrip(oracle, L, T, seed=9, sid=2, rank=rank, world=world)
        M, E = sweep_strips([strip], TorchDistExchange(), L, n, rec)
        rows = torch.from_numpy(strip.buf[1:strip.n + 1].copy())
        parts = [None] * world
        dist.all_gather_object(parts, (strip.r0, rows.numpy()))
        if rank == 0:
            full = np.concatenate([p[1] for p in sorted(parts, key=lambda z: z[0])])
            q.put((M, E, full))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,L", [(2, 64), (3, 70), (4, 96)])
def test_strips_over_gloo_ranks_equal_whole_lattice(orc, world, L):
    T, n, rec = 2.269185, 6, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, L, T, n, rec, q), nprocs=world, join=True,
                       start_method="spawn")
    M, E, full = q.get(timeout=60)
    s = orc.init_hot(L, 9, 2)
    thr4, thr8 = orc.thresholds(T)
    Mo, Eo = orc.run(s, n, 9, 2, thr4, thr8)
    assert np.array_equal(full, s)
    assert M == [int(v) for v in Mo[rec - 1::rec]] and E == [int(v) for v in Eo[rec - 1::rec]]


def test_lpt_partition_balances_and_covers():
    from paper_1007_3726_gb300.distributed import lpt_partition

    work = [256 ** 2 * 10000] * 32 + [512 ** 2 * 10000] * 32 + [1024 ** 2 * 10000] * 32 + \
           [2048 ** 2 * 10000] * 32
    for world in (1, 2, 3, 4, 8):
        parts = lpt_partition(work, world)
        assert sorted(i for p in parts for i in p) == list(range(len(work)))
        loads = [sum(work[i] for i in p) for p in parts]
        # LPT: the heaviest rank exceeds the mean by at most the largest job
        assert max(loads) - sum(work) / world <= max(work)
    # 5 -> rank 0, 4 -> rank 1, 2 -> rank 1 (4 < 5), 1 -> rank 0 (5 < 6)
    assert lpt_partition([5, 1, 4, 2], 2) == [[0, 1], [2, 3]]
    with pytest.raises(ValueError):
        lpt_partition([1], 0)


def _oracle_runner(specs):
    import oracle

    out = []
    for sp in specs:
        thr4, thr8 = oracle.thresholds(sp["T"])
        s = oracle.init_hot(sp["L"], sp["seed"], sp["stream_id"])
        M, E = oracle.run(s, sp["sweeps"], sp["seed"], sp["stream_id"], thr4, thr8)
        out.append((M.tolist(), E.tolist(), s.tobytes()))
    return out


def _sharded_worker(rank, world, port, specs, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1007_3726_gb300.distributed import run_sharded

        res = run_sharded(specs, _oracle_runner)
        if rank == 0:
            q.put(res)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_lattices_over_gloo_ranks_equal_one_rank(orc, world):
    """Independent lattices of uneven size split over gloo ranks by LPT: every
    lattice's samples and final state equal the one-rank run."""
    rng = np.random.default_rng(5)
    specs = [dict(L=int(L), T=float(rng.uniform(1.8, 3.0)), seed=3, stream_id=i, sweeps=int(rng.integers(3, 9)))
             for i, L in enumerate([8, 16, 24, 8, 32, 12, 16, 40, 8])]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    mp.start_processes(_sharded_worker, args=(world, port, specs, q), nprocs=world, join=True,
                       start_method="spawn")
    got = q.get(timeout=60)
    assert got == _oracle_runner(specs)
