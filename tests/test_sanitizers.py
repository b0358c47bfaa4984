"""Host-side memory and undefined-behaviour checks (AddressSanitizer and
UndefinedBehaviorSanitizer), the CPU substitute for a device memory checker:
the oracle and the host code of libising are rebuilt with the sanitizers into
a temporary folder and exercised in a child process with the sanitizer
runtimes preloaded.  Any report fails the test; the sanitized oracle must also
compute exactly what the normal build computes.  No GPU is used."""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-fsanitize=address,undefined", "-fno-omit-frame-pointer", "-fno-sanitize-recover=undefined"]


def _runtime(name):
    p = subprocess.run(["gcc", "-print-file-name=" + name], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


def _env(**extra):
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("gcc's sanitizer runtimes are not installed")
    env = dict(os.environ, LD_PRELOAD=asan + ":" + ubsan,
               ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1", PYTHONPATH=ROOT)
    env.update(extra)
    return env


def _check(r):
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "AddressSanitizer" not in out and "runtime error" not in out, out[-4000:]
    return r.stdout


ORACLE_SCRIPT = r"""
import json, os, numpy as np, oracle
assert not os.environ.get("LD_PRELOAD") or "libasan" in open("/proc/self/maps").read()
L, T, seed, sid = 24, 2.269185, 7, 3
thr4, thr8 = oracle.thresholds(T)
s = oracle.init_hot(L, seed, sid)
M, E = oracle.run(s, 6, seed, sid, thr4, thr8, check=True)
w = oracle.init_hot(64, seed, sid, row0=10, nrows=20)
oracle.run_window(w, 64, 10, 3, seed, sid, thr4, thr8)
Mt, Et = oracle.cold_tiled_counts(64, 2, seed, sid, thr4, thr8, up=True, tile_rows=16)
f = oracle.init_hot(16, seed, sid)
Mf, Ef = oracle.run_field(f, 4, seed, sid, T, 0.3)
ft, fa = oracle.field_thresholds(T, 0.3)
mo = oracle.moments(M, E, N=L * L, T=T)
ph = oracle.philox(np.arange(40, dtype=np.uint32).reshape(10, 4), [[1, 2]])
print(json.dumps({"M": M.tolist(), "E": E.tolist(), "s": s.sum().item(), "w": w.tobytes().hex(),
                  "Mt": Mt.tolist(), "Et": Et.tolist(), "Mf": Mf.tolist(), "Ef": Ef.tolist(),
                  "ft": ft.tolist(), "mo": mo, "ph": ph.tolist()}))
"""


def test_oracle_under_asan_and_ubsan(tmp_path):
    lib = tmp_path / "libising_oracle_san.so"
    subprocess.run(["gcc", "-O1", "-g", "-fopenmp", "-shared", "-fPIC", *SAN, "-o", str(lib),
                    os.path.join(ROOT, "oracle", "ising_oracle.c"), "-lm"], check=True)
    san = _check(subprocess.run([sys.executable, "-c", ORACLE_SCRIPT], capture_output=True, text=True,
                                env=_env(ISING_ORACLE_LIB=str(lib), OMP_NUM_THREADS="2"), cwd=ROOT))
    plain = subprocess.run([sys.executable, "-c", ORACLE_SCRIPT], capture_output=True, text=True,
                           env=dict(os.environ, PYTHONPATH=ROOT), cwd=ROOT, check=True).stdout
    assert san.strip().splitlines()[-1] == plain.strip().splitlines()[-1]


ABI_SCRIPT = r"""
import sys, numpy as np
import paper_1007_3726_gb300 as P
P.load(sys.argv[1])
maps = open("/proc/self/maps").read()
assert "libasan" in maps and "libising_san" in maps
assert P.thresholds(2.269185) == (736899708, 126431970)
for T in (0.01, 1.0, 2.0, 50.0, 1e300):
    P.thresholds(T)
for bad in (0.0, -1.0, float("nan"), float("inf")):
    try:
        P.thresholds(bad)
        raise SystemExit("accepted T=%r" % bad)
    except P.IsingError:
        pass
thr, alw = P.ising_field_thresholds(2.0, 0.7)
assert P.ising_strip_observables(64, 4096, 0) == (4096, -8192)
for args in ((1, 0, 0), (64, 5000, 0), (64, 0, 9000)):
    try:
        P.ising_strip_observables(*args)
        raise SystemExit("accepted %r" % (args,))
    except P.IsingError:
        pass
n = P.ising_launch_candidates(1024)
assert len(n) > 60
for L in (0, 63, 100, 2 ** 21):
    try:
        P.Lattice(L, 2.0)
        raise SystemExit("accepted L=%d" % L)
    except P.IsingError:
        pass
try:
    P.ising_sweep_noalloc(0, 64, 32, 2.0, 1, 0, 0, 1, 0)
    raise SystemExit("accepted a null lattice")
except P.IsingError:
    pass
print("ok", P.ising_last_error())
"""


def test_host_library_under_asan_and_ubsan(tmp_path):
    """The host code of libising (validation, thresholds, launch candidates,
    error paths) rebuilt with the sanitizers; without a GPU the calls that
    would launch a kernel fail cleanly before any device work."""
    from paper_1007_3726_gb300 import _build

    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    # one -Xcompiler per flag: nvcc splits its argument at commas
    host = []
    for f in ["-fPIC", "-O1", "-g", "-fsanitize=address", "-fsanitize=undefined", "-fno-omit-frame-pointer",
              "-fno-sanitize-recover=undefined"]:
        host += ["-Xcompiler", f]
    objs = []

    def compile_one(src):
        obj = str(tmp_path / (os.path.basename(src) + ".o"))
        cmd = [nvcc, *_build.ARCH, "-O1", "-std=c++17", "-I", _build.INCLUDE, "-I", _build.CSRC, *host,
               "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-3000:]
        return obj

    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        objs = list(ex.map(compile_one, _build._sources()))
    lib = str(tmp_path / "libising_san.so")
    r = subprocess.run([nvcc, *_build.ARCH, "-shared", "-o", lib, *objs, "-lpthread", "-lasan", "-lubsan"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = _check(subprocess.run([sys.executable, "-c", ABI_SCRIPT, lib], capture_output=True, text=True,
                                env=_env(CUDA_VISIBLE_DEVICES=""), cwd=ROOT))
    assert out.startswith("ok")
