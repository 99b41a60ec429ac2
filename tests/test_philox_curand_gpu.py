"""Pin: the oracle's Philox4x32-10 (written from Salmon et al., SC'11) equals cuRAND's
curand_Philox4x32_10 word for word.

cuRAND is an independent library implementation of the same generator: with
curand_init(seed, subsequence, offset) the first block curand4 returns is
Philox4x32-10(counter = (offset/4 lo, offset/4 hi, subsequence lo, subsequence hi),
key = (seed lo, seed hi)), which is exactly the oracle's keying of the AWGN
stream (counter = (p, ue_id, rx)).  The probe is compiled here with nvcc.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_philox_matches_curand():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    rng = np.random.default_rng(1)
    cases = [(0, 0, 0), (0x77170002, 3 | (1 << 32), 4 * 12345), ((1 << 64) - 1, (1 << 64) - 1, 0),
             (0x123456789ABCDEF0, 7, 4 * ((1 << 33) + 5))]
    cases += [(int(rng.integers(0, 1 << 63)), int(rng.integers(0, 1 << 40)), 4 * int(rng.integers(0, 1 << 40)))
              for _ in range(60)]
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "probe")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                        os.path.join(HERE, "cuda", "philox_curand_probe.cu"), "-o", exe], check=True)
        inp = "".join(f"{s} {q} {o}\n" for s, q, o in cases)
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (seed, sub, off), line in zip(cases, out):
        got = [int(w, 16) for w in line.split()]
        p = off // 4
        ctr = [p & 0xFFFFFFFF, p >> 32, sub & 0xFFFFFFFF, sub >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        assert list(oracle.philox4x32_10(ctr, key)) == got, (seed, sub, off)
