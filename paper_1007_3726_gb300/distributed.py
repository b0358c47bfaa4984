"""One lattice over several ranks (GPUs) as row strips, after the paper's
super-lattice decomposition with border exchange (Sec. 6.1), reduced to 1-D:
rank r holds global rows [L r / R, L (r + 1) / R) with a halo row above and
below.  Before every checkerboard step the ranks swap boundary rows with their
two ring neighbours (one row of L/8 bytes each way), then every rank updates
its strip (ising_strip_step); at recorded sweeps the per-rank step-B counts
are summed (an int64 all-reduce).  Because the random draws are keyed by global
site indices, the lattice and every sample are identical to the one-GPU run
for any number of ranks.

The exchange is pluggable: `TorchDistExchange` uses torch.distributed (NCCL on
GPUs, gloo on CPUs), `LocalExchange` moves rows between strips held by one
process (ranks emulated on one GPU).  The strip object only needs
`boundary_rows()`, `set_halos()`, `step()`, `zero_counts()` and `counts()`.
"""
from __future__ import annotations


def strip_rows(L: int, rank: int, world: int) -> tuple[int, int]:
    """(first global row, number of rows) of a rank's strip."""
    r0 = L * rank // world
    r1 = L * (rank + 1) // world
    return r0, r1 - r0


class LocalExchange:
    """Halo exchange among strips held by one process (ring order = list order)."""

    def fill_halos(self, strips):
        tops = [s.boundary_rows()[0].clone() for s in strips]
        bots = [s.boundary_rows()[1].clone() for s in strips]
        n = len(strips)
        for k, s in enumerate(strips):
            s.set_halos(bots[(k - 1) % n], tops[(k + 1) % n])

    def sum_counts(self, strips):
        tot = None
        for s in strips:
            c = s.counts()
            tot = c.clone() if tot is None else tot + c
        return tot


class TorchDistExchange:
    """Halo exchange over torch.distributed: one strip per process, ranks in a ring.

    Every rank posts, in this order, send(bottom row -> rank below), send(top row
    -> rank above), recv(top halo <- rank above), recv(bottom halo <- rank below),
    with tags; NCCL matches a pair's messages in posting order, gloo by tag, and
    both pair each row with the right halo even when the two neighbours are the
    same rank."""

    TAG_DOWN, TAG_UP = 11, 12

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def fill_halos(self, strips):
        (s,) = strips
        top, bot = s.boundary_rows()
        if self.world == 1:
            s.set_halos(bot, top)
            return
        dist = self.dist
        up = (self.rank - 1) % self.world
        down = (self.rank + 1) % self.world
        g = self.group
        gu = dist.get_global_rank(g, up) if g is not None else up
        gd = dist.get_global_rank(g, down) if g is not None else down
        top_halo = top.clone()
        bot_halo = bot.clone()
        ops = [dist.P2POp(dist.isend, bot.contiguous(), gd, g, self.TAG_DOWN),
               dist.P2POp(dist.isend, top.contiguous(), gu, g, self.TAG_UP),
               dist.P2POp(dist.irecv, top_halo, gu, g, self.TAG_DOWN),
               dist.P2POp(dist.irecv, bot_halo, gd, g, self.TAG_UP)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        s.set_halos(top_halo, bot_halo)

    def sum_counts(self, strips):
        (s,) = strips
        c = s.counts().clone()
        self.dist.all_reduce(c, op=self.dist.ReduceOp.SUM, group=self.group)
        return c


def sweep_strips(strips, exchange, L: int, nsweeps: int, record_every: int = 0):
    """Sweeps the strips (all at the same sweep index) and returns the (M, E)
    samples of the whole lattice at the recorded sweeps."""
    from . import ising_strip_observables

    Ms, Es = [], []
    for _ in range(nsweeps):
        t = strips[0].t
        rec = record_every and (t + 1) % record_every == 0
        if rec:
            for s in strips:
                s.zero_counts()
        for p in (0, 1):
            exchange.fill_halos(strips)
            for s in strips:
                s.step(p, count=bool(rec and p == 1))
        for s in strips:
            s.t += 1
        if rec:
            c = exchange.sum_counts(strips).cpu()
            M, E = ising_strip_observables(L, int(c[0]), int(c[1]))
            Ms.append(M)
            Es.append(E)
    return Ms, Es


class StripLattice:
    """A rank's strip of an L x L lattice on the GPU (packed words, ising_strip_*)."""

    def __init__(self, L: int, T: float, seed: int = 0, stream_id: int = 0, init: str = "hot",
                 rank: int = 0, world: int = 1, word_bits: int = 64, device=None):
        import torch

        from . import ising_strip_init, load

        load()
        self.L, self.T, self.seed, self.stream_id = L, T, seed, stream_id
        self.word_bits = word_bits
        self.row0, self.nrows = strip_rows(L, rank, world)
        dt = torch.int64 if word_bits == 64 else torch.int32
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.buf = torch.zeros((self.nrows + 2, L // word_bits), dtype=dt, device=dev)
        self._counts = torch.zeros(2, dtype=torch.int64, device=dev)
        self.t = 0
        self._stream = torch.cuda.current_stream(dev)
        ising_strip_init(self.buf.data_ptr(), L, word_bits, self.row0, self.nrows, init, seed, stream_id,
                         self._stream)

    def boundary_rows(self):
        return self.buf[1], self.buf[self.nrows]

    def set_halos(self, top, bottom):
        self.buf[0].copy_(top)
        self.buf[self.nrows + 1].copy_(bottom)

    def step(self, p: int, count: bool = False):
        from . import ising_strip_step

        ising_strip_step(self.buf.data_ptr(), self.L, self.word_bits, self.row0, self.nrows, self.T,
                         self.seed, self.stream_id, self.t, p,
                         self._counts.data_ptr() if count else None, self._stream)

    def zero_counts(self):
        self._counts.zero_()

    def counts(self):
        return self._counts

    def rows(self):
        """The strip's packed rows (without halos)."""
        return self.buf[1:self.nrows + 1]


# ---------------------------------------------------- independent lattices --
def lpt_partition(work, world: int) -> list[list[int]]:
    """Longest-processing-time split of independent jobs over `world` ranks: the
    jobs in order of decreasing work (ties by index), each to the rank with the
    least work so far (ties to the lowest rank).  Returns each rank's job
    indices in increasing order.  Deterministic, so every rank computes the same
    split without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(work)), key=lambda k: (-work[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += work[i]
    return [sorted(p) for p in parts]


def run_sharded(specs, runner, group=None):
    """Runs independent lattices (or requests) spread over the ranks of a
    torch.distributed group by lpt_partition of their work L^2 x sweeps:
    runner(list of specs) runs one rank's share and returns one result per
    spec; the results of all ranks are gathered on every rank and returned in
    the order of `specs`.  A lattice's results depend only on its own seed,
    stream and sweeps, so they equal a one-rank run of the same specs.  With
    no initialised process group the call runs everything on this process."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return list(runner(list(specs)))
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    parts = lpt_partition([int(s["L"]) ** 2 * int(s["sweeps"]) for s in specs], world)
    mine = parts[rank]
    res = list(runner([specs[i] for i in mine]))
    if len(res) != len(mine):
        raise RuntimeError("runner returned %d results for %d specs" % (len(res), len(mine)))
    gathered = [None] * world
    dist.all_gather_object(gathered, list(zip(mine, res)), group=group)
    out = [None] * len(specs)
    for chunk in gathered:
        for i, r in chunk:
            out[i] = r
    return out


def batch_runner(record_every: int, batch_opts=None):
    """A runner for run_sharded on this rank's GPU: the specs' lattices in one
    persistent batch launch; each result is the lattice's samples (M, E) and
    its FP64 moments."""

    def run(specs):
        from . import Batch, Lattice

        if not specs:
            return []
        keys = ("L", "T", "seed", "stream_id", "init", "word_bits")
        lats = [Lattice(**{k: sp[k] for k in keys if k in sp}) for sp in specs]
        with Batch(lats, [sp["sweeps"] for sp in specs], record_every, **(batch_opts or {})) as b:
            b.run(1)
        out = []
        for lat in lats:
            M, E = lat.samples()
            out.append({"M": M, "E": E, "obs": lat.measure()})
            lat.close()
        return out

    return run
