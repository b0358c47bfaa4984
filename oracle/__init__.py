"""Oracle for the checkerboard Metropolis sweep of the 2D Ising model (arXiv:1007.3726).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path (the
CUDA library in ``paper_1007_3726_gb300``) never touches it, and it shares no
code with that path: this package holds its own Philox4x32-10, thresholds, one
byte per spin lattice and bookkeeping (``ising_oracle.c``), plus exact
references (``exact.py``).

The C code is built with gcc into ``oracle/libising_oracle.so`` by ``build()``
and loaded here through ctypes; every function below is a thin marshalling
wrapper.  See the header of ``ising_oracle.c`` for the passages of the paper
each function follows and for the site/counter contract.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(``tests/test_oracle_*.py``): Philox against Triton's CPU interpreter, the
thresholds against 60-digit arithmetic, the update rule against exact flip
probabilities and exact 4x4 / 6x6 Boltzmann averages, the bookkeeping against
recounts, the moments against hand-summed closed forms.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ising_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libising_oracle.so")
_lock = threading.Lock()
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i8p = ctypes.POINTER(ctypes.c_int8)
_dblp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ising_oracle.c with gcc (OpenMP) into libising_oracle.so."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # ISING_ORACLE_LIB: another build of ising_oracle.c (the sanitizer tests)
    lib = ctypes.CDLL(os.environ.get("ISING_ORACLE_LIB") or build())
    lib.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    lib.orc_philox_batch.argtypes = [ctypes.c_uint64, _u32p, _u32p, _u32p]
    lib.orc_thresholds.argtypes = [ctypes.c_double, _u32p, _u32p]
    lib.orc_thresholds.restype = ctypes.c_int
    lib.orc_init_hot.argtypes = [_i8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                 ctypes.c_uint64, ctypes.c_uint32]
    lib.orc_init_cold.argtypes = [_i8p, ctypes.c_uint64, ctypes.c_int]
    lib.orc_recount.argtypes = [_i8p, ctypes.c_uint64, _i64p, _i64p]
    lib.orc_half_sweep.argtypes = [_i8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint32, _i64p, _i64p]
    lib.orc_run.argtypes = [_i8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                            ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                            _i64p, _i64p, _i64p, _i64p, ctypes.c_int]
    lib.orc_run.restype = ctypes.c_int
    lib.orc_run_window.argtypes = [_i8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
    lib.orc_cold_tiled_counts.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_uint32, _i64p, _i64p]
    lib.orc_cold_tiled_counts.restype = ctypes.c_int
    lib.orc_half_sweep_field.argtypes = [_i8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                         ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                         ctypes.c_double, _i64p, _i64p]
    lib.orc_run_field.argtypes = [_i8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                  ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                  _i64p, _i64p, _i64p, _i64p, ctypes.c_int]
    lib.orc_run_field.restype = ctypes.c_int
    lib.orc_field_thresholds.argtypes = [ctypes.c_double, ctypes.c_double, _u32p,
                                         ctypes.POINTER(ctypes.c_uint8)]
    lib.orc_field_thresholds.restype = ctypes.c_int
    lib.orc_moments.argtypes = [_i64p, _i64p, ctypes.c_uint64, ctypes.c_uint64,
                                ctypes.c_double, ctypes.c_double, _dblp]
    lib.orc_moments.restype = ctypes.c_uint64
    _lib = lib
    return lib


def _ptr(a: np.ndarray, ctype):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ---------------------------------------------------------------- Philox -------
def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters ``ctr`` (n x 4 uint32) under keys ``key`` (n x 2)."""
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, dtype=np.uint32).reshape(-1, 2),
                                               (ctr.shape[0], 2)))
    out = np.zeros_like(ctr)
    _load().orc_philox_batch(ctr.shape[0], _ptr(ctr, ctypes.c_uint32),
                             _ptr(key, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


# ------------------------------------------------------------ thresholds -------
def thresholds(T: float) -> tuple[int, int]:
    """(thr4, thr8) = floor(2^32 exp(-dE/T)) for dE = 4, 8 (Sec. 3)."""
    t4 = ctypes.c_uint32()
    t8 = ctypes.c_uint32()
    if _load().orc_thresholds(float(T), ctypes.byref(t4), ctypes.byref(t8)) != 0:
        raise ValueError("temperature must be finite and positive: %r" % (T,))
    return int(t4.value), int(t8.value)


# --------------------------------------------------------------- lattices ------
def init_hot(L: int, seed: int, stream_id: int = 0, row0: int = 0, nrows: int | None = None):
    """Hot start (i.i.d. +-1 with p = 1/2 from Philox) of rows [row0, row0+nrows)."""
    nrows = L if nrows is None else nrows
    s = np.empty((nrows, L), dtype=np.int8)
    _load().orc_init_hot(_ptr(s, ctypes.c_int8), L, row0, nrows, seed, stream_id)
    return s


def init_cold(L: int, value: int = 1) -> np.ndarray:
    s = np.empty((L, L), dtype=np.int8)
    _load().orc_init_cold(_ptr(s, ctypes.c_int8), s.size, int(value))
    return s


def recount(s: np.ndarray) -> tuple[int, int]:
    """Full recount (M, E) of a periodic L x L int8 lattice."""
    L = s.shape[0]
    assert s.shape == (L, L) and s.dtype == np.int8
    s = np.ascontiguousarray(s)
    M = ctypes.c_int64()
    E = ctypes.c_int64()
    _load().orc_recount(_ptr(s, ctypes.c_int8), L, ctypes.byref(M), ctypes.byref(E))
    return int(M.value), int(E.value)


def half_sweep(s: np.ndarray, t: int, p: int, seed: int, stream_id: int, thr4: int, thr8: int,
               L: int | None = None, row0: int = 0, periodic: bool = True):
    """One checkerboard step in place; returns the incremental (dM, dE)."""
    L = s.shape[1] if L is None else L
    assert s.dtype == np.int8 and s.flags.c_contiguous and s.shape[1] == L
    dM = ctypes.c_int64()
    dE = ctypes.c_int64()
    _load().orc_half_sweep(_ptr(s, ctypes.c_int8), L, row0, s.shape[0], 1 if periodic else 0,
                           t, p, seed, stream_id, thr4, thr8, ctypes.byref(dM), ctypes.byref(dE))
    return int(dM.value), int(dE.value)


def run(s: np.ndarray, nsweeps: int, seed: int, stream_id: int, thr4: int, thr8: int,
        t0: int = 0, check: bool = True, M0=None, E0=None):
    """Sweeps t0 .. t0+nsweeps-1 in place on a periodic lattice.

    Returns (M, E) int64 arrays after each sweep.  With ``check`` the incremental
    bookkeeping is compared with a full recount after every sweep and a mismatch
    raises AssertionError.
    """
    L = s.shape[0]
    assert s.shape == (L, L) and s.dtype == np.int8 and s.flags.c_contiguous
    if M0 is None or E0 is None:
        M0, E0 = recount(s)
    m = ctypes.c_int64(M0)
    e = ctypes.c_int64(E0)
    M = np.zeros(nsweeps, dtype=np.int64)
    E = np.zeros(nsweeps, dtype=np.int64)
    rc = _load().orc_run(_ptr(s, ctypes.c_int8), L, t0, nsweeps, seed, stream_id, thr4, thr8,
                         ctypes.byref(m), ctypes.byref(e), _ptr(M, ctypes.c_int64),
                         _ptr(E, ctypes.c_int64), 1 if check else 0)
    if rc != 0:
        raise AssertionError("incremental M/E differ from the recount after sweep %d" % (t0 + rc - 1))
    return M, E


def run_window(s: np.ndarray, L: int, row0: int, nsweeps: int, seed: int, stream_id: int,
               thr4: int, thr8: int, t0: int = 0):
    """Light-cone run on rows [row0, row0 + s.shape[0]) of an L x L lattice, in place.

    After k sweeps the buffer rows 2k .. nrows-1-2k equal the periodic lattice's.
    """
    assert s.dtype == np.int8 and s.flags.c_contiguous and s.shape[1] == L
    _load().orc_run_window(_ptr(s, ctypes.c_int8), L, row0, s.shape[0], t0, nsweeps, seed,
                           stream_id, thr4, thr8)


def cold_tiled_counts(L: int, k: int, seed: int, stream_id: int, thr4: int, thr8: int,
                      up: bool = True, tile_rows: int = 1024):
    """M, E of the whole L x L lattice after each of its first k sweeps from a cold
    start, tile by tile in light-cone windows (no L x L array is held)."""
    M = np.zeros(k, dtype=np.int64)
    E = np.zeros(k, dtype=np.int64)
    rc = _load().orc_cold_tiled_counts(L, 1 if up else 0, k, tile_rows, seed, stream_id, thr4, thr8,
                                       _ptr(M, ctypes.c_int64), _ptr(E, ctypes.c_int64))
    if rc != 0:
        raise ValueError("tile_rows must divide L and leave room for the margins (%d)" % rc)
    return M, E


# ------------------------------------------------------------ field H != 0 ---
def field_thresholds(T: float, H: float):
    """(thr, always): 10 thresholds and always-accept flags indexed 5 i + c, with i = 0
    for S = -1 and 1 for S = +1 and c the number of anti-aligned neighbours."""
    thr = np.zeros(10, dtype=np.uint32)
    alw = np.zeros(10, dtype=np.uint8)
    if _load().orc_field_thresholds(float(T), float(H), _ptr(thr, ctypes.c_uint32),
                                    _ptr(alw, ctypes.c_uint8)) != 0:
        raise ValueError("T must be finite and positive and H finite: %r, %r" % (T, H))
    return thr, alw.astype(bool)


def half_sweep_field(s: np.ndarray, t: int, p: int, seed: int, stream_id: int, T: float, H: float):
    """One checkerboard step in a field H, in place on a periodic lattice;
    returns the incremental (dM, dE_bond)."""
    L = s.shape[0]
    assert s.shape == (L, L) and s.dtype == np.int8 and s.flags.c_contiguous
    dM = ctypes.c_int64()
    dE = ctypes.c_int64()
    _load().orc_half_sweep_field(_ptr(s, ctypes.c_int8), L, t, p, seed, stream_id, float(T), float(H),
                                 ctypes.byref(dM), ctypes.byref(dE))
    return int(dM.value), int(dE.value)


def run_field(s: np.ndarray, nsweeps: int, seed: int, stream_id: int, T: float, H: float,
              t0: int = 0, check: bool = True, M0=None, E0=None):
    """Sweeps t0 .. t0+nsweeps-1 in a field H, in place; returns (M, E_bond) after each."""
    L = s.shape[0]
    assert s.shape == (L, L) and s.dtype == np.int8 and s.flags.c_contiguous
    if M0 is None or E0 is None:
        M0, E0 = recount(s)
    m = ctypes.c_int64(M0)
    e = ctypes.c_int64(E0)
    M = np.zeros(nsweeps, dtype=np.int64)
    E = np.zeros(nsweeps, dtype=np.int64)
    rc = _load().orc_run_field(_ptr(s, ctypes.c_int8), L, t0, nsweeps, seed, stream_id, float(T),
                               float(H), ctypes.byref(m), ctypes.byref(e), _ptr(M, ctypes.c_int64),
                               _ptr(E, ctypes.c_int64), 1 if check else 0)
    if rc != 0:
        raise AssertionError("incremental M/E differ from the recount after sweep %d" % (t0 + rc - 1))
    return M, E


MOMENT_NAMES = ("mean_m", "mean_abs_m", "mean_m2", "mean_m4", "mean_e", "mean_e2", "U4", "chi", "C")


def moments(M, E, N: int, T: float, burn: int = 0) -> dict:
    """FP64 observables of integer samples, plain summation in sample order."""
    M = np.ascontiguousarray(np.asarray(M, dtype=np.int64))
    E = np.ascontiguousarray(np.asarray(E, dtype=np.int64))
    assert M.shape == E.shape
    out = np.zeros(9, dtype=np.float64)
    k = _load().orc_moments(_ptr(M, ctypes.c_int64), _ptr(E, ctypes.c_int64), M.size, burn,
                            float(N), float(T), _ptr(out, ctypes.c_double))
    d = dict(zip(MOMENT_NAMES, out.tolist()))
    d["n_samples"] = int(k)
    return d
