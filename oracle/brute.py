"""Exact rational brute force for tiny inputs -- TEST INFRASTRUCTURE ONLY.

Independent of tt_oracle.c: written symbol by symbol in Python integers and
``fractions.Fraction`` so every product and sum is exact.  It follows the same
definition (Sec. III-B, y_u = x * h_u with the UE's time-varying response
sampled from its trace, Sec. IV), but walks the slot structure instead of
searching for the symbol of each sample, and evaluates the trace-time
interpolation exactly.  No AWGN (noise is pinned statistically instead).
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Sequence

import numpy as np


def _frac(v) -> Fraction:
    return Fraction(float(v))          # float32 -> exact binary fraction


def _trace_entry(taps, i: int, loop: bool):
    n = taps.shape[0]
    return taps[i % n] if loop else taps[min(i, n - 1)]


def anchor_exact(taps: np.ndarray, a_start: int, a: int, step_samples, loop: bool):
    """Exact H[a] ([n_rx][n_tx][K] of complex Fractions as (re, im) pairs).

    ``a_start`` is the first sample of symbol a; step_samples == 0 means one entry per symbol.
    """
    def cplx(v):
        return (_frac(v.real), _frac(v.imag))

    if not step_samples:
        e = _trace_entry(taps, a, loop)
        return [[[cplx(e[r, t, k]) for k in range(e.shape[2])] for t in range(e.shape[1])]
                for r in range(e.shape[0])]
    p = Fraction(a_start) / Fraction(step_samples)
    i0 = p.numerator // p.denominator
    f = p - i0
    e0, e1 = _trace_entry(taps, i0, loop), _trace_entry(taps, i0 + 1, loop)
    out = []
    for r in range(e0.shape[0]):
        row = []
        for t in range(e0.shape[1]):
            col = []
            for k in range(e0.shape[2]):
                a0, a1 = cplx(e0[r, t, k]), cplx(e1[r, t, k])
                col.append((a0[0] + f * (a1[0] - a0[0]), a0[1] + f * (a1[1] - a0[1])))
            row.append(col)
        out.append(row)
    return out


def keep_top_n(H, top_n: int):
    """Sparse convolution (Sec. III-C): per link, the top_n taps of |H[a]|^2, ties to the lower
    index, the powers compared exactly (Fractions)."""
    n_rx, n_tx, K = len(H), len(H[0]), len(H[0][0])
    keep = [[[True] * K for _ in range(n_tx)] for _ in range(n_rx)]
    if not top_n or top_n >= K:
        return keep
    for r in range(n_rx):
        for t in range(n_tx):
            p = [H[r][t][k][0] ** 2 + H[r][t][k][1] ** 2 for k in range(K)]
            for k in range(K):
                beat = sum(1 for j in range(K) if p[j] > p[k] or (p[j] == p[k] and j < k))
                keep[r][t][k] = beat < top_n
    return keep


def run_exact(symbol_len: Sequence[int], delays: Sequence[int], taps: np.ndarray, x: np.ndarray,
              s_first: int = 0, step_samples=0, loop: bool = False, top_n: int = 0):
    """Exact y (lists of Fraction pairs) and packed q for slots s_first.. of one UE.

    x: int16 [n_tx][n_slots*N][2]; taps: complex [T][n_rx][n_tx][K].  top_n > 0 keeps, for each
    symbol and link, only the top_n taps of the symbol's anchor (Sec. III-C sparse convolution).
    Returns (y, q) with y[r][i] = (re, im) Fractions and q int16 [n_rx][n_slots*N][2].
    """
    L = list(symbol_len)
    n = sum(L)
    n_tx, total = x.shape[0], x.shape[1]
    n_rx = taps.shape[1]
    n_slots = total // n
    xs = [[(int(x[t, i, 0]), int(x[t, i, 1])) for i in range(total)] for t in range(n_tx)]
    y: List[List] = [[None] * total for _ in range(n_rx)]
    for sl in range(n_slots):
        s = s_first + sl
        b_local = 0
        for j, Lj in enumerate(L):
            a = s * len(L) + j
            b_abs = s * n + b_local
            nxt_abs = b_abs + Lj                     # first sample of anchor a+1
            H0 = anchor_exact(taps, b_abs, a, step_samples, loop)
            H1 = anchor_exact(taps, nxt_abs, a + 1, step_samples, loop)
            keep = keep_top_n(H0, top_n)
            for off in range(Lj):
                i = sl * n + b_local + off           # index inside the processed block
                tau = Fraction(off, Lj)
                for r in range(n_rx):
                    acc_re = Fraction(0)
                    acc_im = Fraction(0)
                    for t in range(n_tx):
                        for k, d in enumerate(delays):
                            src = i - int(d)
                            if src < 0 or not keep[r][t][k]:
                                continue
                            h0, h1 = H0[r][t][k], H1[r][t][k]
                            hr = h0[0] + tau * (h1[0] - h0[0])
                            hi = h0[1] + tau * (h1[1] - h0[1])
                            xr, xi = xs[t][src]
                            acc_re += hr * xr - hi * xi
                            acc_im += hr * xi + hi * xr
                    y[r][i] = (acc_re, acc_im)
            b_local += Lj
    q = np.zeros((n_rx, total, 2), dtype=np.int16)
    for r in range(n_rx):
        for i in range(total):
            for c in range(2):
                v = round(y[r][i][c])               # Fraction.__round__: ties to even
                q[r, i, c] = max(-32768, min(32767, v))
    return y, q


def to_complex(y) -> np.ndarray:
    return np.array([[complex(float(v[0]), float(v[1])) for v in row] for row in y])
