"""Pins of the oracle's Philox4x32-10 (SC'11 description) against a library routine.

The Philox4x32-10 that Triton ships (``tl.philox``), run on the CPU by Triton's
interpreter, is an implementation independent of the oracle; the two must agree
on every counter word and key word.  The interpreter has to be switched on before
Triton is imported, so it runs in a child process.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

_CHILD = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def _philox_kernel(out, c0p, c1p, c2p, c3p, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c0p + i); c1 = tl.load(c1p + i); c2 = tl.load(c2p + i); c3 = tl.load(c3p + i)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out + i * 4 + 0, a); tl.store(out + i * 4 + 1, b)
    tl.store(out + i * 4 + 2, c); tl.store(out + i * 4 + 3, d)

req = json.loads(sys.stdin.read())
res = []
for seed, ctrs in req:
    ctr = np.array(ctrs, dtype=np.uint64).reshape(-1, 4)
    n = ctr.shape[0]
    cols = [torch.from_numpy(ctr[:, i].astype(np.int64)).to(torch.uint32) for i in range(4)]
    out = torch.zeros(4 * n, dtype=torch.uint32)
    _philox_kernel[(1,)](out, *cols, seed, N=n)
    res.append(out.to(torch.int64).tolist())
print(json.dumps(res))
"""


def _triton_philox(cases):
    pytest.importorskip("triton")
    env = dict(os.environ)
    env["TRITON_INTERPRET"] = "1"
    proc = subprocess.run([sys.executable, "-c", _CHILD], input=json.dumps(cases), env=env,
                          capture_output=True, text=True, timeout=600)
    assert proc.returncode == 0, proc.stderr[-2000:]
    return [np.array(r, dtype=np.uint64).astype(np.uint32).reshape(-1, 4) for r in json.loads(proc.stdout)]


def test_philox_matches_triton_interpreter(orc):
    rng = np.random.default_rng(20100720)
    cases = []
    # random counters under random 64-bit keys
    for _ in range(4):
        seed = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        ctr = rng.integers(0, 2 ** 32, size=(64, 4), dtype=np.uint64)
        cases.append((seed, ctr.tolist()))
    # the counters the sweep actually uses: (g, 0, t, stream<<1 | p) and the hot start's
    ctr = []
    for g in (0, 1, 2, 3, 1023, 2 ** 31, 2 ** 32 - 1):
        for t in (0, 1, 999, 2 ** 32 - 2):
            for c3 in (0, 1, 2 * 95 + 1, 2 ** 32 - 1):
                ctr.append([g, 0, t, c3])
    ctr += [[5, 3, 0xFFFFFFFF, 0], [0, 0, 0, 0], [0xFFFFFFFF] * 4]
    ctr += rng.integers(0, 2 ** 32, size=(128 - len(ctr), 4), dtype=np.uint64).tolist()
    cases.append((7, ctr))
    cases.append((0, ctr))
    cases.append((2 ** 64 - 1, ctr[:64]))
    want = _triton_philox(cases)
    for (seed, c), w in zip(cases, want):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        got = orc.philox(np.array(c, dtype=np.uint64).astype(np.uint32), key)
        assert np.array_equal(got, w), (seed, c[:2])


def test_philox_output_bits_are_balanced(orc):
    # 2^16 consecutive counters: every output bit is set about half the time
    g = np.arange(1 << 16, dtype=np.uint32)
    ctr = np.stack([g, np.zeros_like(g), np.full_like(g, 3), np.full_like(g, 1)], axis=1)
    out = orc.philox(ctr, [1, 0])
    bits = ((out[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1, 128)
    frac = bits.mean(axis=0)
    sigma = 0.5 / np.sqrt(bits.shape[0])
    assert np.all(np.abs(frac - 0.5) < 5.5 * sigma)
