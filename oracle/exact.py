"""Exact references for the 2D Ising model (J = 1, periodic boundaries, field H).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``enumerate_averages(L, T, H=0)`` - brute force over all 2^(L*L) states (L <= 4):
  the plain definition of the Boltzmann averages of the Hamiltonian of Sec. 3,
  Eq. 1, weight exp(-(E - H M)/T) with E the bond energy.
* ``transfer_averages(L, T, H=0)`` - the same averages by a row-to-row transfer
  matrix that keeps the magnetisation distribution (any L up to about 8).
* ``onsager_tc()``, ``onsager_m0(T)``, ``onsager_u(T)`` - Onsager's exact
  critical temperature (quoted as T_C ~ 2.269185 in Sec. 1), spontaneous
  magnetisation and energy per spin of the infinite lattice.
* ``flip_probabilities(s, p, thr4, thr8)`` - exact probability that each site
  flips in one checkerboard step from state ``s`` (Sec. 3 acceptance rule with
  integer thresholds).
* ``metropolis_probabilities(s, p, T, H)`` - the same in a field, from the real
  Metropolis factor min(1, exp(-dE/T)) with dE = 2 S (sum_n S_n + H).
"""
from __future__ import annotations

import math

import numpy as np


# ------------------------------------------------------------ brute force ----
def _energy_mag_all_states(L: int):
    n = L * L
    idx = np.arange(1 << n, dtype=np.int64)
    bits = ((idx[:, None] >> np.arange(n, dtype=np.int64)[None, :]) & 1).astype(np.int8)
    s = (2 * bits - 1).reshape(-1, L, L).astype(np.int32)
    M = s.sum(axis=(1, 2))
    E = -(s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) - (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    return E.astype(np.int64), M.astype(np.int64)


def _averages_from_weights(E, M, logw, N, T):
    logw = logw - logw.max()
    w = np.exp(logw)
    Z = w.sum()
    m = M / N
    e = E / N
    out = {
        "mean_m": float((w * m).sum() / Z),
        "mean_e": float((w * e).sum() / Z),
        "mean_e2": float((w * e * e).sum() / Z),
        "mean_abs_m": float((w * np.abs(m)).sum() / Z),
        "mean_m2": float((w * m * m).sum() / Z),
        "mean_m4": float((w * m ** 4).sum() / Z),
    }
    out["U4"] = 1.0 - out["mean_m4"] / (3.0 * out["mean_m2"] ** 2)
    return out


def enumerate_averages(L: int, T: float, H: float = 0.0) -> dict:
    """Exact averages of m, e = E/N (bond energy), |m|, m^2, m^4 for an L x L
    periodic lattice in a field H, L <= 4."""
    assert L * L <= 20
    E, M = _energy_mag_all_states(L)
    return _averages_from_weights(E.astype(np.float64), M.astype(np.float64), -(E - H * M) / T,
                                  L * L, T)


# -------------------------------------------------------- transfer matrix ----
def _row_tables(L: int):
    r = np.arange(1 << L, dtype=np.int64)
    bits = ((r[:, None] >> np.arange(L)[None, :]) & 1).astype(np.int64)
    spins = 2 * bits - 1                                   # (2^L, L)
    m_row = spins.sum(axis=1)                              # magnetisation of a row
    e_row = -(spins * np.roll(spins, -1, axis=1)).sum(axis=1)   # horizontal bonds in a row
    e_vert = -(spins @ spins.T)                            # vertical bonds between two rows
    return m_row, e_row, e_vert


def density_of_states(L: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Exact g(E, M) of the L x L periodic lattice (L even) by a row transfer matrix.

    Rows are added one at a time.  For every first row r0 the partial sums
    A[r, E, M] count the configurations of the rows so far whose last row is r;
    adding row rn adds the vertical bonds between r and rn, the horizontal bonds
    inside rn and the magnetisation of rn.  Closing the torus adds the vertical
    bonds between the last row and r0.  Returns (E_values, M_values, g) with
    g[i, k] the number of states with energy E_values[i] and magnetisation
    M_values[k] (float64 holding exact integers up to 2^53).
    """
    assert L % 2 == 0 and L >= 2
    m_row, e_row, e_vert = _row_tables(L)
    R = 1 << L
    N = L * L
    nE = 2 * N + 1            # index (E + 2N) / 2
    nM = N + 1                # index (M + N) / 2
    vvals = np.unique(e_vert)
    masks = [(e_vert == v).astype(np.float64) for v in vvals]      # [r, rn]
    g = np.zeros((nE, nM))
    for r0 in range(R):
        A = np.zeros((R, nE, nM))
        A[r0, (e_row[r0] + 2 * N) // 2, (m_row[r0] + N) // 2] = 1.0
        for _ in range(L - 1):
            flat = A.reshape(R, -1)
            B = np.zeros_like(A)
            for v, Iv in zip(vvals, masks):
                C = (Iv.T @ flat).reshape(R, nE, nM)
                B += np.roll(C, int(v) // 2, axis=1)
            for rn in range(R):
                B[rn] = np.roll(np.roll(B[rn], int(e_row[rn]) // 2, axis=0), int(m_row[rn]) // 2, axis=1)
            A = B
        for r in range(R):
            g += np.roll(A[r], int(e_vert[r, r0]) // 2, axis=0)
    E_vals = 2 * np.arange(nE) - 2 * N
    M_vals = 2 * np.arange(nM) - N
    return E_vals, M_vals, g


def transfer_averages(L: int, T: float, H: float = 0.0) -> dict:
    """Exact averages in a field H from the density of states g(E, M)."""
    E_vals, M_vals, g = density_of_states(L)
    ii, kk = np.nonzero(g)
    E = E_vals[ii].astype(np.float64)
    M = M_vals[kk].astype(np.float64)
    logw = np.log(g[ii, kk]) - (E - H * M) / T
    return _averages_from_weights(E, M, logw, L * L, T)


# ------------------------------------------------------------------ Onsager --
def onsager_tc() -> float:
    """T_c = 2 / ln(1 + sqrt 2) (J = k_B = 1)."""
    return 2.0 / math.log(1.0 + math.sqrt(2.0))


def onsager_m0(T: float) -> float:
    """Spontaneous magnetisation per spin (1 - sinh(2/T)^-4)^(1/8) below T_c, else 0."""
    if T >= onsager_tc():
        return 0.0
    return (1.0 - math.sinh(2.0 / T) ** -4) ** 0.125


def onsager_u(T: float) -> float:
    """Energy per spin of the infinite lattice (textbook closed form with K(kappa))."""
    from scipy.special import ellipk

    b = 1.0 / T
    kappa = 2.0 * math.sinh(2 * b) / math.cosh(2 * b) ** 2
    K = ellipk(kappa * kappa)            # scipy's ellipk takes the parameter m = k^2
    return -(1.0 / math.tanh(2 * b)) * (1.0 + (2.0 / math.pi) * (2.0 * math.tanh(2 * b) ** 2 - 1.0) * K)


# --------------------------------------------------- one-step probabilities --
def flip_probabilities(s: np.ndarray, p: int, thr4: int, thr8: int) -> np.ndarray:
    """Probability that each site of ``s`` flips in the checkerboard step of parity p.

    Sites of the other parity never flip.  A site of parity p with energy
    change dE = 2 S sum_n S_n flips with probability 1 if dE <= 0, thr4 / 2^32
    if dE = 4 and thr8 / 2^32 if dE = 8.
    """
    L = s.shape[0]
    s = s.astype(np.int64)
    nsum = np.roll(s, 1, 0) + np.roll(s, -1, 0) + np.roll(s, 1, 1) + np.roll(s, -1, 1)
    dE = 2 * s * nsum
    prob = np.where(dE <= 0, 1.0, np.where(dE == 4, thr4 / 2.0 ** 32, thr8 / 2.0 ** 32))
    y, x = np.indices((L, L))
    return np.where(((x + y) & 1) == p, prob, 0.0)


def metropolis_probabilities(s: np.ndarray, p: int, T: float, H: float) -> np.ndarray:
    """Probability that each site of ``s`` flips in the checkerboard step of parity p
    in a field H: min(1, exp(-dE/T)) with dE = 2 S (sum_n S_n + H) for the sites of
    parity p (Sec. 3), 0 for the others.  Real numbers, not the integer thresholds:
    they differ from thr / 2^32 by less than 2^-32."""
    L = s.shape[0]
    s = s.astype(np.float64)
    nsum = np.roll(s, 1, 0) + np.roll(s, -1, 0) + np.roll(s, 1, 1) + np.roll(s, -1, 1)
    dE = 2.0 * s * (nsum + H)
    prob = np.where(dE <= 0, 1.0, np.exp(-np.maximum(dE, 0.0) / T))
    y, x = np.indices((L, L))
    return np.where(((x + y) & 1) == p, prob, 0.0)
