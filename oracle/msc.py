"""The paper's CPU multi-spin-coding program (Sec. 4) with a Boltzmann-pattern
pool: a second, faster timed CPU baseline.

TEST INFRASTRUCTURE AND CPU BASELINE ONLY (tests/ and bench.py's CPU baseline).
Not bit-exact with the GPU library or the oracle: it draws one pool address per
32-spin word, as the paper does, instead of one Philox draw per site, so it is
pinned statistically (tests/test_msc_pool.py).  The C code is msc_pool.c,
built with gcc (OpenMP over rows) into oracle/libising_msc.so.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msc_pool.c")
_LIB_PATH = os.path.join(_HERE, "libising_msc.so")
_lock = threading.Lock()
_lib = None
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.msc_pool_fill.argtypes = [_u32p, _u32p, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64]
        lib.msc_pool_fill.restype = ctypes.c_int
        lib.msc_sweeps.argtypes = [_u32p, ctypes.c_uint64, _u32p, _u32p, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_uint64, ctypes.c_uint64, _i64p, _i64p]
        lib.msc_sweeps.restype = ctypes.c_int
        lib.msc_recount.argtypes = [_u32p, ctypes.c_uint64, _i64p, _i64p]
        _lib = lib
    return _lib


def _p(a, t):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(t))


class Pool:
    """npool (a power of two) Boltzmann pattern pairs (exp4, exp8) at T."""

    def __init__(self, T: float, npool: int = 1 << 22, seed: int = 1):
        if npool <= 0 or npool & (npool - 1):
            raise ValueError("npool must be a power of two")
        self.T, self.npool = T, npool
        self.exp4 = np.zeros(npool, dtype=np.uint32)
        self.exp8 = np.zeros(npool, dtype=np.uint32)
        if _load().msc_pool_fill(_p(self.exp4, ctypes.c_uint32), _p(self.exp8, ctypes.c_uint32), npool,
                                 float(T), seed) != 0:
            raise ValueError("T must be finite and positive")


def pack(spins: np.ndarray) -> np.ndarray:
    """int8 +1/-1 (L x L) -> L x L/32 words, bit b of word w = x = 32 w + b."""
    bits = (np.ascontiguousarray(spins) > 0).astype(np.uint8)
    return np.packbits(bits, axis=1, bitorder="little").view(np.uint32).copy()


def unpack(lat: np.ndarray) -> np.ndarray:
    b = np.unpackbits(np.ascontiguousarray(lat).view(np.uint8), axis=1, bitorder="little")
    return b.astype(np.int8) * 2 - 1


def sweeps(lat: np.ndarray, pool: Pool, n: int, seed: int, t0: int = 0, record: bool = True):
    """n sweeps in place on a packed lattice; (M, E) after each sweep if record."""
    L = lat.shape[0]
    M = np.zeros(max(n, 1), dtype=np.int64) if record else None
    E = np.zeros(max(n, 1), dtype=np.int64) if record else None
    rc = _load().msc_sweeps(_p(lat, ctypes.c_uint32), L, _p(pool.exp4, ctypes.c_uint32),
                            _p(pool.exp8, ctypes.c_uint32), pool.npool, t0, n, seed,
                            _p(M, ctypes.c_int64) if record else None, _p(E, ctypes.c_int64) if record else None)
    if rc != 0:
        raise ValueError("L must be a multiple of 32")
    return (M[:n], E[:n]) if record else None


def recount(lat: np.ndarray) -> tuple[int, int]:
    M = ctypes.c_int64()
    E = ctypes.c_int64()
    _load().msc_recount(_p(lat, ctypes.c_uint32), lat.shape[0], ctypes.byref(M), ctypes.byref(E))
    return int(M.value), int(E.value)
