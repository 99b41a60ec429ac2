"""Pin on the CPU: the oracle's Philox4x32-10 (written from Salmon et al., SC'11) equals
Triton's ``tl.philox`` word for word.

Triton's generator is a separate library implementation of the same counter-based
generator, shipped as Python source and run here by Triton's CPU interpreter
(``tests/philox_triton_words.py``, in a child process).  Together with the GPU test against
cuRAND it fixes the raw word stream that the AWGN of the convolution draws from: a wrong
multiplier, Weyl constant, round count, word order or key half fails it.  Triton is used by
this test only; the product path has no Triton code.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _cases():
    rng = np.random.default_rng(20250108)
    ctr, key = [], []
    m = 0xFFFFFFFF
    # edge counters and keys: zero, all ones, single bits in each word, each key half alone
    for c in ([0, 0, 0, 0], [m, m, m, m], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1],
              [1 << 31, 0, 0, 0], [0, 0, 0, 1 << 31]):
        for k in ([0, 0], [m, m], [1, 0], [0, 1]):
            ctr.append(c)
            key.append(k)
    # the AWGN keying: counter (sample block lo, hi, UE, Rx antenna), key (seed lo, seed hi)
    for p, ue, rx in ((0, 0, 0), (12345, 3, 1), ((1 << 33) + 5, 511, 3), ((1 << 40) - 1, 7, 0)):
        ctr.append([p & m, p >> 32, ue, rx])
        key.append([0x77170002, 0])
    for _ in range(200):
        ctr.append([int(v) for v in rng.integers(0, 1 << 32, size=4, dtype=np.uint64)])
        key.append([int(v) for v in rng.integers(0, 1 << 32, size=2, dtype=np.uint64)])
    return ctr, key


def test_oracle_philox_matches_triton_library_words():
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    ctr, key = _cases()
    env = dict(os.environ, TRITON_INTERPRET="1")
    res = subprocess.run([sys.executable, os.path.join(HERE, "philox_triton_words.py")],
                         input=json.dumps({"ctr": ctr, "key": key}), capture_output=True, text=True,
                         env=env, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    got = np.asarray(json.loads(res.stdout), dtype=np.uint64)
    want = np.array([oracle.philox4x32_10(c, k) for c, k in zip(ctr, key)], dtype=np.uint64)
    assert got.shape == want.shape == (len(ctr), 4)
    bad = np.nonzero(np.any(got != want, axis=1))[0]
    assert bad.size == 0, [(ctr[i], key[i], got[i].tolist(), want[i].tolist()) for i in bad[:4]]
