"""Finite-size scaling of the Binder cumulant (Sec. 3, Eq. 2): the paper tests its
implementation by locating T_c where the U4(T) curves of different lattice sizes
cross.

`run_fss` simulates every (L, T) of a grid in one persistent batch, drops the
equilibration samples, and returns U4 with block-bootstrap errors (the samples of
a Markov chain are correlated: blocks longer than the autocorrelation time are
resampled).  `crossings` interpolates where the curves of consecutive sizes cross,
with bootstrap errors.  Each U4 is the library's (ising_measure_from: FP64 sums
of the exact integer samples in sample order); only the bootstrap replicas,
which resample blocks of those samples, are formed here.
"""
from __future__ import annotations

import numpy as np


def bootstrap_binder(M: np.ndarray, N: float, nblocks: int = 50, nboot: int = 200, rng=None):
    """Block-bootstrap replicas of U4 (nboot values) from the samples M."""
    rng = np.random.default_rng(0) if rng is None else rng
    m = M.astype(np.float64) / N
    n = (len(m) // nblocks) * nblocks
    blocks = m[:n].reshape(nblocks, -1)
    b2 = np.mean(blocks ** 2, axis=1)
    b4 = np.mean(blocks ** 4, axis=1)
    reps = np.empty(nboot)
    for i in range(nboot):
        k = rng.integers(0, nblocks, size=nblocks)
        s2, s4 = b2[k].mean(), b4[k].mean()
        reps[i] = 1.0 - s4 / (3.0 * s2 * s2)
    return reps


def run_fss(Ls=(64, 128, 256, 512), temps=None, sweeps=200000, record_every=10, burn_frac=0.2,
            seed=3, init="cold_up", batch_opts=None):
    """U4(L, T) from one persistent batch; returns {L: (temps, U4, U4_boot[nboot, nT])}.

    `sweeps` is one count for every size or a {L: sweeps} map (critical slowing
    down: the autocorrelation time of the Metropolis update grows about as
    L^2.17 at T_c, so larger lattices need more sweeps)."""
    import paper_1007_3726_gb300 as P

    if temps is None:
        temps = np.linspace(2.24, 2.30, 32)
    per_L = sweeps if isinstance(sweeps, dict) else {L: sweeps for L in Ls}
    lats, keys, ns = [], [], []
    for iL, L in enumerate(Ls):
        for iT, T in enumerate(temps):
            lats.append(P.Lattice(L, float(T), seed=seed, stream_id=64 * iL + iT, init=init))
            keys.append((L, iT))
            ns.append(int(per_L[L]))
    opts = dict(batch_opts or {})
    with P.Batch(lats, ns, record_every, **opts) as b:
        b.run(1)
    out = {}
    rng = np.random.default_rng(12345)
    for (L, iT), lat in zip(keys, lats):
        burn = int(burn_frac * per_L[L] / record_every)
        M, _ = lat.samples(first=burn)
        u = lat.measure(first_sample=burn)["U4"]
        reps = bootstrap_binder(M, float(L) * L, rng=rng)
        d = out.setdefault(L, [np.asarray(temps, dtype=np.float64), np.zeros(len(temps)),
                               np.zeros((len(reps), len(temps)))])
        d[1][iT] = u
        d[2][:, iT] = reps
        lat.close()
    return {L: tuple(v) for L, v in out.items()}


def _cross(T, a, b):
    d = a - b
    for i in range(len(T) - 1):
        if d[i] == 0:
            return float(T[i])
        if d[i] * d[i + 1] < 0:
            return float(T[i] + (T[i + 1] - T[i]) * d[i] / (d[i] - d[i + 1]))
    return None


def crossings(res: dict):
    """T where U4 of consecutive sizes cross, with the bootstrap standard error."""
    Ls = sorted(res)
    out = []
    for L1, L2 in zip(Ls[:-1], Ls[1:]):
        T, u1, b1 = res[L1]
        _, u2, b2 = res[L2]
        c = _cross(T, u1, u2)
        reps = [x for x in (_cross(T, b1[i], b2[i]) for i in range(len(b1))) if x is not None]
        err = float(np.std(reps, ddof=1)) if len(reps) > 2 else None
        out.append({"L1": L1, "L2": L2, "T_cross": c, "err": err, "n_boot": len(reps)})
    return out
