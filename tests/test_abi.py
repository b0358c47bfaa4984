"""The C-ABI library builds, loads and exports every symbol declared in include/*.h,
and its host-only logic (thresholds, validation, errors) behaves as declared.
No compute call is made here, so these run without a GPU."""
import ctypes
import glob
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and
                                not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="needs nvcc to build libising")


@pytest.fixture(scope="module")
def ising():
    import paper_1007_3726_gb300 as P

    P.build()
    P.load()
    return P


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\bISING_API\b[^;{]*?\b(ising_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_core_entry_points():
    names = _declared_functions()
    for core in ("ising_create", "ising_sweep", "ising_measure", "ising_destroy"):
        assert core in names
    assert len(names) >= 12


def test_library_exports_every_declared_symbol(ising):
    lib = ctypes.CDLL(ising.LIB_PATH)
    missing = [n for n in sorted(_declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_library_exports_nothing_else(ising):
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", ising.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported <= _declared_functions(), exported - _declared_functions()


def test_library_thresholds_equal_oracle(ising, orc):
    rng = np.random.default_rng(1)
    temps = [0.01, 0.5, 1.0, 1.5, 2.0, 2.2, 2.246493, 2.269185, 2.35, 3.5, 1e300]
    temps += list(rng.uniform(0.2, 20.0, size=500))
    for T in temps:
        assert ising.ising_thresholds(float(T)) == orc.thresholds(float(T)), T
    # the published configurations' values
    assert ising.ising_thresholds(2.269185) == (736899708, 126431970)
    assert ising.ising_thresholds(2.0) == (581260615, 78665070)


@pytest.mark.parametrize("bad", [0.0, -2.0, float("nan"), float("inf")])
def test_library_rejects_bad_temperature(ising, bad):
    with pytest.raises(ising.IsingError) as ei:
        ising.ising_thresholds(bad)
    assert ei.value.status == ising.ERR_INVALID
    assert "finite" in ising.ising_last_error()


@pytest.mark.parametrize("field,value", [("L", 0), ("L", 32), ("L", 100), ("L", 2 ** 21),
                                         ("T", -1.0), ("T", float("nan")),
                                         ("H", float("nan")), ("H", float("-inf")),
                                         ("stream_id", 2 ** 31), ("word_bits", 16),
                                         ("init", 9), ("init", 3)])
def test_create_validates_before_touching_the_gpu(ising, field, value):
    p = ising.IsingParams(L=256, T=2.0, seed=1, stream_id=0, init=2, init_data=None, word_bits=0)
    setattr(p, field, value)
    h = ctypes.c_void_p(123)
    st = ising.load().ising_create(ctypes.byref(p), None, ctypes.byref(h))
    assert st == ising.ERR_INVALID
    assert h.value is None
    assert ising.ising_last_error() != ""


def test_library_field_thresholds_equal_oracle(ising, orc):
    """The ten class thresholds of the field update (Eq. 1 with H != 0) are the
    oracle's, and H = 0 reduces them to (thr8, thr4) at c = 0, 1."""
    rng = np.random.default_rng(2)
    cases = [(T, H) for T in (0.01, 0.7, 2.0, 2.269185, 3.5, 1e300)
             for H in (0.0, 1e-300, 0.1, -0.1, 1.0, 2.0, -2.0, 4.0, 5.5, -1e3)]
    cases += list(zip(rng.uniform(0.2, 20.0, 300), rng.uniform(-6.0, 6.0, 300)))
    for T, H in cases:
        thr, alw = ising.ising_field_thresholds(float(T), float(H))
        othr, oalw = orc.field_thresholds(float(T), float(H))
        assert np.array_equal(thr, othr) and np.array_equal(alw, oalw), (T, H)
    thr4, thr8 = ising.ising_thresholds(2.269185)
    thr, alw = ising.ising_field_thresholds(2.269185, 0.0)
    assert list(thr) == [thr8, thr4, 0, 0, 0] * 2
    assert list(alw) == [False, False, True, True, True] * 2
    for bad in ((0.0, 0.0), (1.0, float("nan")), (float("inf"), 0.0)):
        with pytest.raises(ising.IsingError):
            ising.ising_field_thresholds(*bad)


def test_null_handles_and_arguments(ising):
    lib = ising.load()
    assert lib.ising_destroy(None) == ising.OK
    assert lib.ising_sweep(None, 1, 0, None, None, 0) == ising.ERR_INVALID
    assert lib.ising_measure(None, None) == ising.ERR_INVALID
    assert lib.ising_create(None, None, None) == ising.ERR_INVALID
    assert lib.ising_set_temperature(None, 2.0) == ising.ERR_INVALID
    assert lib.ising_set_field(None, 0.5) == ising.ERR_INVALID
    assert lib.ising_get_params(None, None, None) == ising.ERR_INVALID
    a = ising.ALLOC_FN(lambda n, s, c: None)
    assert lib.ising_set_allocator(a, ctypes.cast(None, ising.FREE_FN), None) == ising.ERR_INVALID


def test_launch_candidates_are_listed_without_a_gpu(ising):
    c = ising.ising_launch_candidates(32768)
    assert len(c) >= 162
    assert {x["proc_bits"] for x in c} == {32, 64}
    assert all(32768 % x["rows_per_item"] == 0 for x in c)
    assert len(ising.ising_launch_candidates(192)) >= 162
    # the one-CTA kernel is a candidate exactly for power-of-two L <= 1024, its
    # warp-specialised forms (block 1024) at L = 64 (grid 1, 2, 4, 8), 128 and
    # 256 (grid 2, 4, 8)
    for L, k, ws in ((64, 40, 4), (128, 39, 3), (256, 39, 3), (512, 36, 0), (1024, 36, 0), (192, 0, 0),
                     (2048, 0, 0), (32768, 0, 0)):
        tiny = [x for x in ising.ising_launch_candidates(L) if x["proc_bits"] == 8]
        assert len(tiny) == k and sum(x["block"] == 1024 for x in tiny) == ws, L
    # L = 2^20: configurations whose item count does not fit 32 bits are left out
    big = ising.ising_launch_candidates(2 ** 20)
    assert 0 < len(big) < len(c)
    for x in big:
        assert (2 ** 20 // x["rows_per_item"]) * (2 ** 20 // x["proc_bits"]) < 2 ** 32
