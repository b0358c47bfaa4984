"""Synthetic workloads (the paper has no dataset; all lattices are synthetic by
definition).  Each function returns the parameters of the lattices of one
workload; nothing here does any of the method's arithmetic.

* plain_L64          L = 64, T = 2.269185, cold start +1, seed 1, 1000 sweeps,
                     M/E every sweep (the smallest case).
* large_L32768       L = 32768 (2^30 spins), hot start seed 7, T = 2.269185,
                     1000 sweeps, M/E every sweep.
* fss_batch          L in {256, 512, 1024, 2048} x 32 temperatures evenly spaced
                     in [2.20, 2.35], hot starts, seed 3, stream 32 * iL + iT,
                     10^4 sweeps, a sample every 10 sweeps (finite-size scaling
                     of the Binder cumulant, Sec. 3 Eq. 2).
* largest_L524288    L = 524288 (2^38 spins, 32 GiB), cold start, T = 2.0,
                     seed 5, 200 sweeps, M/E every sweep.
* paper_benchmark    the paper's Table 1 shape: L = 4096, T = 0.99 T_c, hot start.
* served_requests    a Poisson request stream (see serve.py).
"""
from __future__ import annotations

import math

TC_PRINTED = 2.269185           # Sec. 1
TC_EXACT = 2.0 / math.log(1.0 + math.sqrt(2.0))


def plain_L64():
    return dict(L=64, T=2.269185, seed=1, stream_id=0, init="cold_up", sweeps=1000, record_every=1)


def large_L32768():
    return dict(L=32768, T=2.269185, seed=7, stream_id=0, init="hot", sweeps=1000, record_every=1,
                word_bits=32)


def fss_temperatures(n=32, lo=2.20, hi=2.35):
    return [lo + i * (hi - lo) / (n - 1) for i in range(n)]


def fss_batch(sweeps=10000, record_every=10, Ls=(256, 512, 1024, 2048), ntemps=32):
    out = []
    for iL, L in enumerate(Ls):
        for iT, T in enumerate(fss_temperatures(ntemps)):
            out.append(dict(L=L, T=T, seed=3, stream_id=32 * iL + iT, init="hot", sweeps=sweeps,
                            record_every=record_every))
    return out


def largest_L524288():
    return dict(L=524288, T=2.0, seed=5, stream_id=0, init="cold_up", sweeps=200, record_every=1,
                word_bits=64)


def paper_benchmark(sweeps=1000):
    return dict(L=4096, T=0.99 * TC_PRINTED, seed=11, stream_id=0, init="hot", sweeps=sweeps,
                record_every=1)


def lattice_kwargs(spec: dict) -> dict:
    """The Lattice(...) arguments of a workload entry."""
    keys = ("L", "T", "seed", "stream_id", "init", "word_bits")
    return {k: spec[k] for k in keys if k in spec}


def onsager_m0(T: float) -> float:
    """Onsager's spontaneous magnetisation per spin, (1 - sinh(2/T)^-4)^(1/8) below T_c
    (the reference the L = 524288 workload is compared with)."""
    if T >= TC_EXACT:
        return 0.0
    return (1.0 - math.sinh(2.0 / T) ** -4) ** 0.125
