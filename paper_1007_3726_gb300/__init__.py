"""GB300 (sm_103a) multi-spin-coded checkerboard Metropolis sweep of the 2D Ising
model (after arXiv:1007.3726), behind the C ABI of ``include/ising.h``.

This module is argument marshalling only: every step of the sweep runs in the
CUDA kernels of ``libising.so`` (built in-tree by ``paper_1007_3726_gb300._build``).
There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.

Raw entry points carry the C names (``ising_create``, ``ising_sweep``,
``ising_measure``, ``ising_destroy``, ...); ``Lattice`` wraps one handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB_PATH, build  # noqa: F401

__all__ = [
    "IsingError", "Lattice", "build", "load", "thresholds", "ising_create", "ising_sweep",
    "ising_measure", "ising_measure_from", "ising_destroy", "ising_get_spins", "ising_get_packed", "ising_recount", "ising_get_samples",
    "ising_thresholds", "ising_last_error", "ising_set_allocator", "ising_info",
    "ising_device_spins", "ising_check_guards", "ising_sweep_noalloc", "ising_bench_mix", "ising_strip_init", "ising_strip_step", "ising_strip_observables", "ising_get_launch", "ising_set_launch",
    "ising_launch_candidates", "ising_autotune", "ising_sweep_batch", "ising_batch_tune", "Batch", "Server", "IsingBatchOpts",
    "IsingParams", "IsingLaunch", "IsingObs", "INIT_MODES", "STATUS_NAMES",
]

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_STATE, ERR_CANCELLED = range(7)
STATUS_NAMES = {0: "ISING_OK", 1: "ISING_ERR_INVALID", 2: "ISING_ERR_OOM", 3: "ISING_ERR_CUDA",
                4: "ISING_ERR_TIMEOUT", 5: "ISING_ERR_STATE", 6: "ISING_ERR_CANCELLED"}
INIT_MODES = {"cold_up": 0, "cold": 0, "cold_down": 1, "hot": 2, "buffer": 3, "packed": 4}


class IsingError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class IsingParams(ctypes.Structure):
    _fields_ = [("L", ctypes.c_uint64), ("T", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("stream_id", ctypes.c_uint32), ("init", ctypes.c_int),
                ("init_data", ctypes.c_void_p), ("word_bits", ctypes.c_uint32),
                ("first_sweep", ctypes.c_uint64), ("H", ctypes.c_double)]


class IsingObs(ctypes.Structure):
    _fields_ = [("sweeps_done", ctypes.c_uint64), ("n_samples", ctypes.c_uint64),
                ("M", ctypes.c_int64), ("E", ctypes.c_int64),
                ("mean_m", ctypes.c_double), ("mean_abs_m", ctypes.c_double),
                ("mean_m2", ctypes.c_double), ("mean_m4", ctypes.c_double),
                ("mean_e", ctypes.c_double), ("mean_e2", ctypes.c_double),
                ("U4", ctypes.c_double), ("chi", ctypes.c_double), ("C", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class IsingLaunch(ctypes.Structure):
    _fields_ = [("proc_bits", ctypes.c_uint32), ("regcap", ctypes.c_uint32), ("block", ctypes.c_uint32),
                ("rows_per_item", ctypes.c_uint32), ("grid", ctypes.c_uint32),
                ("insert", ctypes.c_uint32), ("persistent", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class IsingBatchOpts(ctypes.Structure):
    _fields_ = [("block", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("rows_per_item", ctypes.c_uint32), ("insert", ctypes.c_uint32),
                ("use_graph", ctypes.c_uint32), ("wait_ms", ctypes.c_double),
                ("hold_strip", ctypes.c_uint32)]


class IsingServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("epoch_sweeps", ctypes.c_uint32),
                ("max_active", ctypes.c_uint32), ("keep_samples", ctypes.c_uint32),
                ("batch", IsingBatchOpts)]


class IsingRequest(ctypes.Structure):
    _fields_ = [("params", IsingParams), ("nsweeps", ctypes.c_uint64), ("record_every", ctypes.c_uint32),
                ("tag", ctypes.c_uint64)]


class IsingResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int),
                ("obs", IsingObs), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_first_run", ctypes.c_double), ("t_finish", ctypes.c_double),
                ("epochs", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "obs"}
        d["obs"] = self.obs.as_dict()
        return d


class IsingServerCounters(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "admitted", "completed", "failed",
                                                 "cancelled", "queued", "resident", "epochs",
                                                 "mem_used", "peak_mem", "attempts")] + \
               [("busy_seconds", ctypes.c_double), ("now", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_vpp = ctypes.POINTER(ctypes.c_void_p)
_szp = ctypes.POINTER(ctypes.c_size_t)


def load(path: str | None = None):
    """Load libising.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError("libising.so is not built (%s); run paper_1007_3726_gb300.build()" % path)
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    sig = {
        "ising_create": ([ctypes.POINTER(IsingParams), ctypes.c_void_p, ctypes.POINTER(H)], ctypes.c_int),
        "ising_sweep": ([H, ctypes.c_uint64, ctypes.c_uint32, _i64p, _i64p, ctypes.c_uint64], ctypes.c_int),
        "ising_measure": ([H, ctypes.POINTER(IsingObs)], ctypes.c_int),
        "ising_measure_from": ([H, ctypes.c_uint64, ctypes.POINTER(IsingObs)], ctypes.c_int),
        "ising_destroy": ([H], ctypes.c_int),
        "ising_get_spins": ([H, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p], ctypes.c_int),
        "ising_get_packed": ([H, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
        "ising_recount": ([H, _i64p, _i64p], ctypes.c_int),
        "ising_get_samples": ([H, ctypes.c_uint64, ctypes.c_uint64, _i64p, _i64p, _u64p], ctypes.c_int),
        "ising_info": ([H, _u32p, _u64p, _u64p], ctypes.c_int),
        "ising_device_spins": ([H, _vpp, _szp], ctypes.c_int),
        "ising_thresholds": ([ctypes.c_double, _u32p, _u32p], ctypes.c_int),
        "ising_last_error": ([], ctypes.c_char_p),
        "ising_set_allocator": ([ALLOC_FN, FREE_FN, ctypes.c_void_p], ctypes.c_int),
        "ising_get_launch": ([H, ctypes.POINTER(IsingLaunch)], ctypes.c_int),
        "ising_set_launch": ([H, ctypes.POINTER(IsingLaunch)], ctypes.c_int),
        "ising_launch_candidates": ([ctypes.c_uint64, ctypes.POINTER(IsingLaunch), ctypes.c_uint32],
                                    ctypes.c_uint32),
        "ising_autotune": ([H, ctypes.c_uint32, ctypes.POINTER(IsingLaunch),
                            ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "ising_batch_create": ([ctypes.POINTER(H), ctypes.c_uint32, _u64p, ctypes.c_uint32,
                                ctypes.POINTER(IsingBatchOpts), ctypes.POINTER(H)], ctypes.c_int),
        "ising_batch_run": ([H, ctypes.c_uint32], ctypes.c_int),
        "ising_batch_info": ([H, _u32p, _u32p, _u32p, _szp], ctypes.c_int),
        "ising_batch_destroy": ([H], ctypes.c_int),
        "ising_sweep_batch": ([ctypes.POINTER(H), ctypes.c_uint32, _u64p, ctypes.c_uint32], ctypes.c_int),
        "ising_batch_tune": ([ctypes.POINTER(H), ctypes.c_uint32, _u64p, ctypes.c_uint32,
                              ctypes.POINTER(IsingBatchOpts), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "ising_server_create": ([ctypes.POINTER(IsingServerOpts), ctypes.POINTER(H)], ctypes.c_int),
        "ising_server_submit": ([H, ctypes.POINTER(IsingRequest), _u64p], ctypes.c_int),
        "ising_server_cancel": ([H, ctypes.c_uint64], ctypes.c_int),
        "ising_server_poll": ([H, ctypes.POINTER(IsingResult), ctypes.c_uint32, _u32p, ctypes.c_double],
                              ctypes.c_int),
        "ising_server_samples": ([H, ctypes.c_uint64, _i64p, _i64p, ctypes.c_uint64, _u64p], ctypes.c_int),
        "ising_server_stats": ([H, ctypes.POINTER(IsingServerCounters)], ctypes.c_int),
        "ising_server_destroy": ([H], ctypes.c_int),
        "ising_strip_init": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                              ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                              ctypes.c_void_p], ctypes.c_int),
        "ising_strip_step": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                              ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                              ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p],
                             ctypes.c_int),
        "ising_field_thresholds": ([ctypes.c_double, ctypes.c_double, _u32p,
                                    ctypes.POINTER(ctypes.c_uint8)], ctypes.c_int),
        "ising_set_temperature": ([H, ctypes.c_double], ctypes.c_int),
        "ising_set_field": ([H, ctypes.c_double], ctypes.c_int),
        "ising_get_params": ([H, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                             ctypes.c_int),
        "ising_check_guards": ([H, _u32p], ctypes.c_int),
        "ising_strip_observables": ([ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _i64p, _i64p],
                                    ctypes.c_int),
        "ising_bench_mix": ([ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), ctypes.c_void_p], ctypes.c_int),
        "ising_sweep_noalloc": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                 ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                 ctypes.c_uint32, _i64p, _i64p, ctypes.c_uint64, ctypes.c_void_p],
                                ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status: int):
    if status != OK:
        raise IsingError(status, ising_last_error())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream / ExternalStream


# ------------------------------------------------------------- raw C names --
def ising_last_error() -> str:
    return load().ising_last_error().decode()


def ising_thresholds(T: float) -> tuple[int, int]:
    a, b = ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().ising_thresholds(float(T), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


thresholds = ising_thresholds


def ising_field_thresholds(T: float, H: float):
    """(thr, always) of the ten classes in a field, index 5 i + c (i = 0 for S = -1)."""
    thr = np.zeros(10, dtype=np.uint32)
    alw = np.zeros(10, dtype=np.uint8)
    _check(load().ising_field_thresholds(float(T), float(H), thr.ctypes.data_as(_u32p),
                                         alw.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
    return thr, alw.astype(bool)


def ising_set_temperature(h, T: float):
    _check(load().ising_set_temperature(h, float(T)))


def ising_set_field(h, H: float):
    _check(load().ising_set_field(h, float(H)))


def ising_get_params(h) -> tuple[float, float]:
    T, H = ctypes.c_double(), ctypes.c_double()
    _check(load().ising_get_params(h, ctypes.byref(T), ctypes.byref(H)))
    return T.value, H.value


def ising_create(params: IsingParams, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().ising_create(ctypes.byref(params), _stream_ptr(stream), ctypes.byref(h)))
    return h


def ising_sweep(h, nsweeps: int, record_every: int = 0, M_out=None, E_out=None, cap: int = 0):
    mp = M_out.ctypes.data_as(_i64p) if M_out is not None else None
    ep = E_out.ctypes.data_as(_i64p) if E_out is not None else None
    _check(load().ising_sweep(h, nsweeps, record_every, mp, ep, cap))


def ising_measure(h) -> dict:
    o = IsingObs()
    _check(load().ising_measure(h, ctypes.byref(o)))
    return o.as_dict()


def ising_measure_from(h, first_sample: int) -> dict:
    o = IsingObs()
    _check(load().ising_measure_from(h, first_sample, ctypes.byref(o)))
    return o.as_dict()


def ising_destroy(h):
    _check(load().ising_destroy(h))


def ising_get_spins(h, row0: int, nrows: int, out: np.ndarray):
    assert out.dtype == np.int8 and out.flags.c_contiguous
    _check(load().ising_get_spins(h, row0, nrows, out.ctypes.data))


def ising_get_packed(h, out: np.ndarray):
    assert out.flags.c_contiguous
    _check(load().ising_get_packed(h, out.ctypes.data, out.nbytes))


def ising_get_samples(h, first: int = 0, count: int | None = None):
    """Recorded (M, E) samples first .. first + count - 1 as int64 arrays."""
    if count is None:
        count = ising_measure(h)["n_samples"] + 1
    M = np.zeros(max(count, 1), dtype=np.int64)
    E = np.zeros(max(count, 1), dtype=np.int64)
    n = ctypes.c_uint64()
    _check(load().ising_get_samples(h, first, count, M.ctypes.data_as(_i64p), E.ctypes.data_as(_i64p),
                                    ctypes.byref(n)))
    return M[:n.value], E[:n.value]


def ising_recount(h) -> tuple[int, int]:
    M, E = ctypes.c_int64(), ctypes.c_int64()
    _check(load().ising_recount(h, ctypes.byref(M), ctypes.byref(E)))
    return M.value, E.value


def ising_info(h) -> tuple[int, int, int]:
    wb, L, sd = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().ising_info(h, ctypes.byref(wb), ctypes.byref(L), ctypes.byref(sd)))
    return wb.value, L.value, sd.value


def ising_device_spins(h) -> tuple[int, int]:
    p, n = ctypes.c_void_p(), ctypes.c_size_t()
    _check(load().ising_device_spins(h, ctypes.byref(p), ctypes.byref(n)))
    return p.value, n.value


def ising_sweep_noalloc(d_spins: int, L: int, word_bits: int, T: float, seed: int, stream_id: int,
                        t0: int, nsweeps: int, record_every: int = 0, M_out=None, E_out=None,
                        cap: int = 0, stream=None):
    """Sweeps on a caller-owned device lattice without any allocation by the
    library (see include/ising.h); M_out / E_out are host int64 arrays of at
    least cap entries (C-contiguous), or both None."""
    for name, arr in (("M_out", M_out), ("E_out", E_out)):
        if arr is None:
            continue
        if not (isinstance(arr, np.ndarray) and arr.dtype == np.int64 and arr.flags.c_contiguous
                and arr.flags.writeable and arr.size >= cap):
            raise ValueError("%s must be a writeable C-contiguous int64 array of at least cap = %d "
                             "entries" % (name, cap))
    mp = M_out.ctypes.data_as(_i64p) if M_out is not None else None
    ep = E_out.ctypes.data_as(_i64p) if E_out is not None else None
    _check(load().ising_sweep_noalloc(d_spins, L, word_bits, float(T), seed, stream_id, t0, nsweeps,
                                      record_every, mp, ep, cap, _stream_ptr(stream)))


def ising_bench_mix(form: int, words_per_thread: int, stream=None) -> tuple[float, float]:
    """The integer-mix microbenchmark (see include/ising.h): (ms, draws per ns)."""
    ms = ctypes.c_double()
    rate = ctypes.c_double()
    _check(load().ising_bench_mix(form, words_per_thread, ctypes.byref(ms), ctypes.byref(rate),
                                  _stream_ptr(stream)))
    return ms.value, rate.value


def ising_get_launch(h) -> dict:
    o = IsingLaunch()
    _check(load().ising_get_launch(h, ctypes.byref(o)))
    return o.as_dict()


def ising_set_launch(h, cfg: dict):
    _check(load().ising_set_launch(h, ctypes.byref(IsingLaunch(**cfg))))


def ising_launch_candidates(L: int) -> list[dict]:
    n = load().ising_launch_candidates(L, None, 0)
    arr = (IsingLaunch * max(n, 1))()
    load().ising_launch_candidates(L, arr, n)
    return [arr[i].as_dict() for i in range(n)]


def ising_autotune(h, reps: int = 3) -> tuple[dict, float]:
    o = IsingLaunch()
    us = ctypes.c_double()
    _check(load().ising_autotune(h, reps, ctypes.byref(o), ctypes.byref(us)))
    return o.as_dict(), us.value


def _handles(lats):
    hs = [(l.handle if isinstance(l, Lattice) else l) for l in lats]
    return (ctypes.c_void_p * len(hs))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in hs])


def ising_sweep_batch(lats, nsweeps, record_every: int = 0):
    """One persistent launch over many lattices (handles or Lattice objects)."""
    arr = _handles(lats)
    ns = (ctypes.c_uint64 * len(lats))(*[int(x) for x in nsweeps])
    _check(load().ising_sweep_batch(arr, len(lats), ns, record_every))


def ising_batch_tune(lats, nsweeps, probe_sweeps: int = 20, **base) -> tuple[dict, float]:
    """Pick batch options by timing probe runs (the lattices are restored)."""
    arr = _handles(lats)
    ns = (ctypes.c_uint64 * len(lats))(*[int(x) for x in nsweeps])
    o = IsingBatchOpts(**base)
    ms = ctypes.c_double()
    _check(load().ising_batch_tune(arr, len(lats), ns, probe_sweeps, ctypes.byref(o), ctypes.byref(ms)))
    return {k: getattr(o, k) for k, _ in IsingBatchOpts._fields_}, ms.value


class Batch:
    """A planned persistent multi-lattice launch (ising_batch_create / _run)."""

    def __init__(self, lats, nsweeps, record_every: int = 0, block: int = 0, ctas_per_sm: int = 0,
                 rows_per_item: int = 0, insert: int = 0, use_graph: bool = False,
                 wait_ms: float = 0.0, hold_strip: int = 0):
        self._lats = list(lats)  # keep the handles alive
        arr = _handles(self._lats)
        ns = (ctypes.c_uint64 * len(self._lats))(*[int(x) for x in nsweeps])
        o = IsingBatchOpts(block=block, ctas_per_sm=ctas_per_sm, rows_per_item=rows_per_item,
                           insert=insert, use_graph=1 if use_graph else 0, wait_ms=wait_ms,
                           hold_strip=hold_strip)
        self._b = ctypes.c_void_p()
        _check(load().ising_batch_create(arr, len(self._lats), ns, record_every, ctypes.byref(o),
                                         ctypes.byref(self._b)))

    def run(self, runs: int = 1):
        _check(load().ising_batch_run(self._b, runs))

    def info(self) -> dict:
        g, b, st, sm = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_size_t()
        _check(load().ising_batch_info(self._b, ctypes.byref(g), ctypes.byref(b), ctypes.byref(st),
                                       ctypes.byref(sm)))
        return {"grid": g.value, "block": b.value, "strips": st.value, "smem_bytes": sm.value}

    def close(self):
        if self._b is not None and self._b.value:
            load().ising_batch_destroy(self._b)
        self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Request server with continuous batching (ising_server_*)."""

    def __init__(self, hbm_budget_bytes: int = 0, epoch_sweeps: int = 0, max_active: int = 0,
                 keep_samples: bool = False, **batch_opts):
        o = IsingServerOpts(hbm_budget_bytes=hbm_budget_bytes, epoch_sweeps=epoch_sweeps,
                            max_active=max_active, keep_samples=1 if keep_samples else 0,
                            batch=IsingBatchOpts(**batch_opts))
        self._s = ctypes.c_void_p()
        _check(load().ising_server_create(ctypes.byref(o), ctypes.byref(self._s)))

    def submit(self, L: int, T: float, nsweeps: int, seed: int = 0, stream_id: int = 0, init: str = "hot",
               record_every: int = 0, word_bits: int = 0, tag: int = 0, H: float = 0.0) -> int:
        p = IsingParams(L=L, T=T, seed=seed, stream_id=stream_id, init=INIT_MODES[init], init_data=None,
                        word_bits=word_bits, H=H)
        r = IsingRequest(params=p, nsweeps=nsweeps, record_every=record_every, tag=tag)
        rid = ctypes.c_uint64()
        _check(load().ising_server_submit(self._s, ctypes.byref(r), ctypes.byref(rid)))
        return rid.value

    def cancel(self, rid: int):
        _check(load().ising_server_cancel(self._s, rid))

    def poll(self, cap: int = 256, wait_s: float = 0.0) -> list[dict]:
        arr = (IsingResult * cap)()
        n = ctypes.c_uint32()
        _check(load().ising_server_poll(self._s, arr, cap, ctypes.byref(n), wait_s))
        return [arr[i].as_dict() for i in range(n.value)]

    def samples(self, rid: int):
        n = ctypes.c_uint64()
        _check(load().ising_server_samples(self._s, rid, None, None, 0, ctypes.byref(n)))
        M = np.zeros(max(n.value, 1), dtype=np.int64)
        E = np.zeros(max(n.value, 1), dtype=np.int64)
        _check(load().ising_server_samples(self._s, rid, M.ctypes.data_as(_i64p), E.ctypes.data_as(_i64p),
                                           n.value, ctypes.byref(n)))
        return M[:n.value], E[:n.value]

    def stats(self) -> dict:
        o = IsingServerCounters()
        _check(load().ising_server_stats(self._s, ctypes.byref(o)))
        return o.as_dict()

    def close(self):
        if self._s is not None and self._s.value:
            load().ising_server_destroy(self._s)
        self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def ising_strip_init(d_rows: int, L: int, word_bits: int, row0: int, nrows: int, init: str = "hot",
                     seed: int = 0, stream_id: int = 0, stream=None):
    _check(load().ising_strip_init(d_rows, L, word_bits, row0, nrows, INIT_MODES[init], seed, stream_id,
                                   _stream_ptr(stream)))


def ising_strip_step(d_rows: int, L: int, word_bits: int, row0: int, nrows: int, T: float, seed: int,
                     stream_id: int, t: int, p: int, d_counts: int | None = None, stream=None):
    _check(load().ising_strip_step(d_rows, L, word_bits, row0, nrows, float(T), seed, stream_id, t, p,
                                   d_counts, _stream_ptr(stream)))


def ising_check_guards(h) -> bool:
    """True while the guard bytes around the handle's lattice are intact."""
    v = ctypes.c_uint32()
    _check(load().ising_check_guards(h, ctypes.byref(v)))
    return bool(v.value)


# guard failures seen when lattices were closed (checked after every GPU test)
guard_failures: list = []


def ising_strip_observables(L: int, n_up: int, n_anti: int) -> tuple[int, int]:
    """(M, E) of an L x L lattice from its summed step-B counts (see include/ising.h)."""
    M = ctypes.c_int64()
    E = ctypes.c_int64()
    _check(load().ising_strip_observables(L, n_up, n_anti, ctypes.byref(M), ctypes.byref(E)))
    return M.value, E.value


_alloc_keepalive = []


def ising_set_allocator(alloc=None, release=None, ctx=None):
    """Install Python callables alloc(bytes, stream) -> int and release(ptr, stream)
    as the library's device allocator (None restores cudaMalloc)."""
    if alloc is None:
        _alloc_keepalive.clear()
        _check(load().ising_set_allocator(ctypes.cast(None, ALLOC_FN), ctypes.cast(None, FREE_FN), None))
        return
    a = ALLOC_FN(lambda n, s, c: alloc(n, s) or None)
    f = FREE_FN(lambda p, s, c: release(p, s))
    _alloc_keepalive[:] = [a, f]
    _check(load().ising_set_allocator(a, f, ctx))


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    import torch

    def alloc(n, s):
        try:
            return torch.cuda.caching_allocator_alloc(n, stream=s or 0)
        except RuntimeError:
            return None

    def release(p, s):
        torch.cuda.caching_allocator_delete(p)

    ising_set_allocator(alloc, release)


# ------------------------------------------------------------------ Lattice --
class Lattice:
    """One simulated lattice (a handle of the C ABI)."""

    def __init__(self, L: int, T: float, seed: int = 0, stream_id: int = 0, init: str = "hot",
                 spins: np.ndarray | None = None, packed: np.ndarray | None = None,
                 word_bits: int = 0, stream=None, first_sweep: int = 0, H: float = 0.0):
        self._h = None
        data = None
        if spins is not None:
            init = "buffer"
            data = np.ascontiguousarray(spins, dtype=np.int8)
            assert data.size == L * L
        elif packed is not None:
            init = "packed"
            data = np.ascontiguousarray(packed)
        self._keep = data
        p = IsingParams(L=L, T=T, seed=seed, stream_id=stream_id, init=INIT_MODES[init],
                        init_data=data.ctypes.data if data is not None else None,
                        word_bits=word_bits, first_sweep=first_sweep, H=H)
        self._h = ising_create(p, stream)
        self._keep = None
        self.L, self.seed, self.stream_id = L, seed, stream_id
        self.word_bits = ising_info(self._h)[0]

    @property
    def handle(self):
        return self._h

    @property
    def T(self) -> float:
        return ising_get_params(self._h)[0]

    @property
    def H(self) -> float:
        return ising_get_params(self._h)[1]

    def set_temperature(self, T: float):
        """New temperature from the next sweep on (annealing)."""
        ising_set_temperature(self._h, T)

    def set_field(self, H: float):
        """New external field from the next sweep on (Eq. 1; 0 = the paper's case)."""
        ising_set_field(self._h, H)

    def sweep(self, nsweeps: int, record_every: int = 0, collect: bool = False):
        """Run sweeps; with collect=True return this call's (M, E) samples."""
        if not collect:
            ising_sweep(self._h, nsweeps, record_every)
            return None
        _, _, done = ising_info(self._h)
        n = (done + nsweeps) // record_every - done // record_every if record_every else 0
        M = np.zeros(max(n, 1), dtype=np.int64)
        E = np.zeros(max(n, 1), dtype=np.int64)
        ising_sweep(self._h, nsweeps, record_every, M, E, n)
        return M[:n], E[:n]

    def measure(self, first_sample: int = 0) -> dict:
        """Counters and FP64 moments of the samples from first_sample on."""
        return ising_measure_from(self._h, first_sample) if first_sample else ising_measure(self._h)

    def spins(self, row0: int = 0, nrows: int | None = None) -> np.ndarray:
        nrows = self.L if nrows is None else nrows
        out = np.empty((nrows, self.L), dtype=np.int8)
        ising_get_spins(self._h, row0, nrows, out)
        return out

    def packed(self) -> np.ndarray:
        dt = np.uint64 if self.word_bits == 64 else np.uint32
        out = np.empty((self.L, self.L // self.word_bits), dtype=dt)
        ising_get_packed(self._h, out)
        return out

    def recount(self) -> tuple[int, int]:
        return ising_recount(self._h)

    def samples(self, first: int = 0, count: int | None = None):
        """All (or some) recorded (M, E) samples of the lattice."""
        return ising_get_samples(self._h, first, count)

    @property
    def launch(self) -> dict:
        return ising_get_launch(self._h)

    def set_launch(self, **cfg):
        """Replace the launch configuration; fields not given keep their current
        values, except that naming proc_bits without persistent means persistent = 0."""
        full = dict(self.launch)
        if "proc_bits" in cfg and "persistent" not in cfg:
            full["persistent"] = 0
        full.update(cfg)
        ising_set_launch(self._h, full)

    def autotune(self, reps: int = 3) -> tuple[dict, float]:
        """Pick the fastest launch configuration (results do not depend on it)."""
        return ising_autotune(self._h, reps)

    def save(self, path: str):
        """Checkpoint: the packed lattice, its parameters, sweep count and samples
        (a .npz file).  Lattice.load(path) resumes it bit for bit: the random
        draws depend only on (seed, stream_id, sweep index, site)."""
        M, E = self.samples()
        np.savez(path, packed=self.packed(), L=self.L, T=self.T, H=self.H, seed=self.seed,
                 stream_id=self.stream_id, word_bits=self.word_bits, sweeps_done=self.sweeps_done,
                 M=M, E=E)

    @classmethod
    def load(cls, path: str, stream=None) -> "Lattice":
        """Resumes a checkpoint written by save().  The samples recorded before the
        checkpoint are returned by `restored_samples`, not counted by measure()."""
        z = np.load(path)
        lat = cls(int(z["L"]), float(z["T"]), seed=int(z["seed"]), stream_id=int(z["stream_id"]),
                  packed=z["packed"], word_bits=int(z["word_bits"]), stream=stream,
                  first_sweep=int(z["sweeps_done"]), H=float(z["H"]) if "H" in z else 0.0)
        lat.restored_samples = (z["M"], z["E"])
        return lat

    @property
    def sweeps_done(self) -> int:
        return ising_info(self._h)[2]

    def guards_intact(self) -> bool:
        return ising_check_guards(self._h)

    def close(self):
        if self._h is not None:
            h, self._h = self._h, None
            try:
                if not ising_check_guards(h):
                    guard_failures.append((self.L, self.seed, self.stream_id))
            except IsingError:
                pass  # a failed handle: its error was reported where it happened
            ising_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
