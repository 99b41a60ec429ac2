"""Philox4x32-10 words from Triton's own ``tl.philox`` (``triton/language/random.py``), run by
Triton's CPU interpreter, as an independent library implementation of Salmon et al. (SC'11).

Test infrastructure only: ``tests/test_philox_library_pin.py`` runs this file in a child
process (``TRITON_INTERPRET=1`` must be set before Triton decides how to run a kernel) and
compares its output with the oracle.  Nothing on the product path uses Triton.

Input on stdin: JSON ``{"ctr": [[c0, c1, c2, c3], ...], "key": [[k0, k1], ...]}`` (one key per
counter).  Output on stdout: JSON list of the four output words per counter.
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_words(ctr_ptr, key_ptr, out_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(ctr_ptr + 4 * i + 0)
    c1 = tl.load(ctr_ptr + 4 * i + 1)
    c2 = tl.load(ctr_ptr + 4 * i + 2)
    c3 = tl.load(ctr_ptr + 4 * i + 3)
    k0 = tl.load(key_ptr + 2 * i + 0).to(tl.uint64)
    k1 = tl.load(key_ptr + 2 * i + 1).to(tl.uint64)
    # tl.philox splits its 64-bit seed into key word 0 (low half) and key word 1 (high half)
    w0, w1, w2, w3 = tl.philox((k1 << 32) | k0, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, w0)
    tl.store(out_ptr + 4 * i + 1, w1)
    tl.store(out_ptr + 4 * i + 2, w2)
    tl.store(out_ptr + 4 * i + 3, w3)


def main() -> None:
    req = json.load(sys.stdin)
    ctr = np.asarray(req["ctr"], dtype=np.uint32).reshape(-1, 4)
    key = np.asarray(req["key"], dtype=np.uint32).reshape(-1, 2)
    n = ctr.shape[0]
    size = 1 << max(0, (n - 1).bit_length())  # tl.arange wants a power of two
    cpad = np.zeros((size, 4), dtype=np.uint32)
    kpad = np.zeros((size, 2), dtype=np.uint32)
    cpad[:n], kpad[:n] = ctr, key
    ct = torch.from_numpy(cpad.reshape(-1).view(np.int32).copy()).view(torch.uint32)
    kt = torch.from_numpy(kpad.reshape(-1).view(np.int32).copy()).view(torch.uint32)
    out = torch.zeros(size * 4, dtype=torch.uint32)
    _philox_words[(1,)](ct, kt, out, N=size)
    words = out.view(torch.int32).numpy().view(np.uint32).reshape(size, 4)[:n]
    json.dump(words.astype(np.uint64).tolist(), sys.stdout)


if __name__ == "__main__":
    main()
