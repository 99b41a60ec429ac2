"""Pins for the FP64 oracle against things other than itself (CPU only).

Each test names what fixes the expected value: exact rational brute force,
a closed form, a library routine for a special case (numpy FFT / convolve /
rint), or a statistical law.  A plausible slip in the oracle (dropped term,
wrong sign, wrong index, transposed operand, off-by-one anchor) fails at least
one of them.
"""
import numpy as np
import pytest

import oracle
from oracle import brute
from tests.helpers import impulse_x, iq_to_complex, nrmse, topn_selections


def _rand_taps(rng, T, n_rx, n_tx, K, scale=1.0):
    z = (rng.standard_normal((T, n_rx, n_tx, K)) + 1j * rng.standard_normal((T, n_rx, n_tx, K))) * scale
    return z.astype(np.complex64)


# --------------------------------------------------------------------------
# 1. exact brute force on tiny inputs (indexing, interpolation, MIMO sums)
# --------------------------------------------------------------------------
CASES = [
    # symbol_len, n_tx, n_rx, delays, n_slots, step_samples, loop
    ([3, 2, 3], 1, 1, [0], 2, 0, False),
    ([3, 2, 3], 1, 1, [0, 1, 5], 3, 0, False),
    ([5, 4, 4, 4], 2, 1, [0, 2, 7, 20], 3, 0, False),        # delay beyond a whole slot
    ([6, 5, 5], 1, 2, [1, 4], 2, 0, True),
    ([4, 4], 2, 2, [0, 3, 9], 4, 5.5, False),                  # trace time steps of 5.5 samples
    ([7, 6, 6, 6], 1, 1, [0, 1, 2, 3], 2, 8.0, True),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_oracle_equals_exact_brute_force(case):
    L, n_tx, n_rx, d, n_slots, step, loop = CASES[case]
    rng = np.random.default_rng(100 + case)
    n = sum(L)
    if step:
        T = int(np.ceil(n_slots * n / step)) + 3
    else:
        T = len(L) * n_slots + 1 if not loop else len(L) + 2
    taps = _rand_taps(rng, T, n_rx, n_tx, len(d))
    x = rng.integers(-3000, 3000, size=(n_tx, n_slots * n, 2)).astype(np.int16)
    for s_first in (0, 3):
        ue = oracle.OracleUE(L, n_tx, n_rx, d, taps, step_samples=step, loop=loop)
        y, q = oracle.run_ue(ue, x, s_first=s_first)
        ye, qe = brute.run_exact(L, d, taps, x, s_first=s_first, step_samples=step, loop=loop)
        ye = brute.to_complex(ye)
        assert nrmse(y, ye) < 1e-13
        assert np.max(np.abs(y - ye)) < 1e-9 * (1 + np.max(np.abs(ye)))
        # packing: identical except where the exact value sits within 1e-9 of a .5 tie
        diff = np.abs(q.astype(np.int32) - qe.astype(np.int32))
        assert diff.max() <= 1
        assert np.count_nonzero(diff) == 0


def test_integer_static_taps_give_exact_int16():
    """Static small-integer taps and integer input: every FP64 step is exact, q matches bit for bit."""
    rng = np.random.default_rng(7)
    L = [9, 7, 7, 7]
    d = [0, 3, 11, 30]
    tap0 = (rng.integers(-3, 4, size=(1, 2, 1, 4)) + 1j * rng.integers(-3, 4, size=(1, 2, 1, 4)))
    taps = np.repeat(tap0, 3 * 4 + 1, axis=0).astype(np.complex64)
    x = rng.integers(-2000, 2000, size=(1, 3 * 30, 2)).astype(np.int16)
    ue = oracle.OracleUE(L, 1, 2, d, taps)
    y, q = oracle.run_ue(ue, x)
    _, qe = brute.run_exact(L, d, taps, x)
    assert np.array_equal(q, qe)
    assert np.all(y.real == np.round(y.real)) and np.all(y.imag == np.round(y.imag))


# --------------------------------------------------------------------------
# 2. unit impulses reproduce taps and delays (closed form)
# --------------------------------------------------------------------------
def test_impulse_reproduces_static_taps_and_delays_across_slots():
    L = [139 * 2] + [137 * 2] * 13         # 5 MHz slot, 3840 samples
    n = sum(L)
    d = np.array([0, 3, 7, 12, 20, 40, 300], dtype=np.int32)
    h = np.array([2 - 1j, -1 + 3j, 4, 1j, -2, 1 + 1j, 3 - 2j], dtype=np.complex64)
    taps = np.tile(h.reshape(1, 1, 1, -1), (14 * 2 + 1, 1, 1, 1))
    ue = oracle.OracleUE(L, 1, 1, d, taps)
    for m0 in (0, 1, n // 2, n - 41, n - 1):           # includes the last sample of slot 0
        x = impulse_x(1, 2 * n, [m0])
        y, q = oracle.run_ue(ue, x)
        a = complex(3, -2)
        expect = np.zeros(2 * n, dtype=np.complex128)
        for dk, hk in zip(d, h):
            if m0 + dk < 2 * n:
                expect[m0 + dk] += a * complex(hk)
        assert np.array_equal(y[0], expect)
        assert np.array_equal(iq_to_complex(q[0]), expect)


def test_impulse_train_follows_linear_ramp_trace():
    """H[a] = (a + 1) * c  =>  h(m) = c * (a + 1 + (m - b_a) / L_a) in closed form."""
    L = [10, 8, 8, 8]
    n = sum(L)
    d = np.array([0, 5], dtype=np.int32)
    c = np.array([1 + 2j, -0.5 + 0.25j])
    T = 4 * 3 + 1
    taps = np.array([[[(a + 1) * c]] for a in range(T)], dtype=np.complex64)
    ue = oracle.OracleUE(L, 1, 1, d, taps)
    starts = np.concatenate([[0], np.cumsum(L)[:-1]])
    for m0 in range(0, 3 * n - 6, 7):
        x = impulse_x(1, 3 * n, [m0], amp=(1, 0))
        y, _ = oracle.run_ue(ue, x)
        for k in range(2):
            m = m0 + d[k]
            s, w = divmod(m, n)
            j = int(np.searchsorted(starts, w, side="right") - 1)
            a = 4 * s + j
            expect = c[k] * (a + 1 + (w - starts[j]) / L[j])
            got = y[0, m] - (y[0, m0] if (k == 1 and d[1] == 0) else 0)
            assert abs(got - expect) < 1e-6 * abs(expect)


# --------------------------------------------------------------------------
# 3. static taps: library convolution (numpy FFT and np.convolve)
# --------------------------------------------------------------------------
def test_static_taps_match_fft_and_convolve():
    rng = np.random.default_rng(3)
    L = [139 * 8] + [137 * 8] * 13          # 20 MHz: 15360 samples per slot
    n = sum(L)
    n_slots = 3
    d = np.sort(np.concatenate([[0], rng.choice(np.arange(1, 257), 23, replace=False)])).astype(np.int32)
    h = (rng.standard_normal(24) + 1j * rng.standard_normal(24)) / np.sqrt(48)
    h = h.astype(np.complex64)
    taps = np.tile(h.reshape(1, 1, 1, -1), (14 * n_slots + 1, 1, 1, 1))
    x = rng.integers(-3000, 3000, size=(1, n_slots * n, 2)).astype(np.int16)
    ue = oracle.OracleUE(L, 1, 1, d, taps)
    y, _ = oracle.run_ue(ue, x)
    xc = iq_to_complex(x[0])
    g = np.zeros(d.max() + 1, dtype=np.complex128)
    g[d] = h.astype(np.complex128)
    nfft = 1 << int(np.ceil(np.log2(len(xc) + len(g))))
    ref = np.fft.ifft(np.fft.fft(xc, nfft) * np.fft.fft(g, nfft))[: len(xc)]
    assert nrmse(y[0], ref) < 1e-12
    ref2 = np.convolve(xc, g)[: len(xc)]
    assert nrmse(y[0], ref2) < 1e-13


def test_mimo_static_is_sum_of_siso_convolutions():
    rng = np.random.default_rng(4)
    L = [6, 5, 5]
    n = sum(L)
    d = np.array([0, 2, 9], dtype=np.int32)
    h = (rng.standard_normal((1, 2, 3, 3)) + 1j * rng.standard_normal((1, 2, 3, 3))).astype(np.complex64)
    taps = np.repeat(h, 3 * 4 + 1, axis=0)
    x = rng.integers(-500, 500, size=(3, 4 * n, 2)).astype(np.int16)
    ue = oracle.OracleUE(L, 3, 2, d, taps)
    y, _ = oracle.run_ue(ue, x)
    for r in range(2):
        ref = np.zeros(4 * n, dtype=np.complex128)
        for t in range(3):
            g = np.zeros(10, dtype=np.complex128)
            g[d] = h[0, r, t].astype(np.complex128)
            ref += np.convolve(iq_to_complex(x[t]), g)[: 4 * n]
        assert nrmse(y[r], ref) < 1e-13


# --------------------------------------------------------------------------
# 4. energy preservation for unit-power taps
# --------------------------------------------------------------------------
def test_unit_power_static_taps_preserve_energy():
    rng = np.random.default_rng(5)
    L = [139 * 16] + [137 * 16] * 13      # 40 MHz
    n = sum(L)
    n_slots = 33                           # ~1e6 samples
    d = np.sort(np.concatenate([[0], rng.choice(np.arange(1, 257), 23, replace=False)])).astype(np.int32)
    p = 10.0 ** (-2.0 * d / d.max())
    p /= p.sum()
    h = np.sqrt(p) * np.exp(2j * np.pi * rng.random(24))
    taps = np.tile(h.astype(np.complex64).reshape(1, 1, 1, -1), (14 * n_slots + 1, 1, 1, 1))
    x = np.clip(np.rint(rng.standard_normal((1, n_slots * n, 2)) * 1024), -32768, 32767).astype(np.int16)
    ue = oracle.OracleUE(L, 1, 1, d, taps)
    y, _ = oracle.run_ue(ue, x, nthreads=0)
    ratio = np.mean(np.abs(y[0, 300:]) ** 2) / np.mean(np.abs(iq_to_complex(x[0])) ** 2)
    assert abs(ratio - 1.0) < 0.02


# --------------------------------------------------------------------------
# 5. single-tap special case (the default rfsim per-symbol scalar fading)
# --------------------------------------------------------------------------
def test_single_tap_is_interpolated_gain_times_input():
    rng = np.random.default_rng(6)
    L = [139 * 2] + [137 * 2] * 13
    n = sum(L)
    n_slots = 2
    T = 14 * n_slots + 1
    a = np.arange(T)
    g = 10.0 ** (-6.0 * (1 - np.cos(2 * np.pi * a / 9.0)) / 20.0)   # periodic fading sanity trace
    taps = (g * np.exp(1j * 0.3 * a)).astype(np.complex64).reshape(T, 1, 1, 1)
    x = rng.integers(-4000, 4000, size=(1, n_slots * n, 2)).astype(np.int16)
    ue = oracle.OracleUE(L, 1, 1, [0], taps)
    y, _ = oracle.run_ue(ue, x)
    starts = np.concatenate([[0], np.cumsum(L)[:-1]])
    xc = iq_to_complex(x[0])
    H = taps[:, 0, 0, 0].astype(np.complex128)
    for m in range(0, n_slots * n, 13):
        s, w = divmod(m, n)
        j = int(np.searchsorted(starts, w, side="right") - 1)
        aa = 14 * s + j
        tau = (w - starts[j]) / L[j]
        h = H[aa] + tau * (H[aa + 1] - H[aa])
        assert abs(y[0, m] - h * xc[m]) <= 1e-9 * (1 + abs(h * xc[m]))


# --------------------------------------------------------------------------
# 6. trace handling: trace-time interpolation, looping, holding
# --------------------------------------------------------------------------
def test_trace_time_interpolation_closed_form():
    """Trace entry i = c * i at sample i*step  =>  H[a] = c * b_a / step exactly (linear in time)."""
    L = [139 * 8] + [137 * 8] * 13
    step = 30720.0 / 7.0                    # not a divisor of anything
    T = 50
    c = np.array([0.5 - 0.25j, 1.0 + 0.125j])
    taps = (np.arange(T)[:, None] * c[None, :]).astype(np.complex64).reshape(T, 1, 1, 2)
    ue = oracle.OracleUE(L, 1, 1, [0, 1], taps, step_samples=step)
    starts = np.concatenate([[0], np.cumsum(L)[:-1]])
    n = sum(L)
    for a in (0, 1, 5, 13, 14, 15, 40, 97):
        b = (a // 14) * n + starts[a % 14]
        H = oracle.anchor(ue, a)[0, 0]
        assert np.allclose(H, c * b / step, rtol=1e-12, atol=1e-12)


def test_trace_loop_and_hold():
    rng = np.random.default_rng(8)
    taps = _rand_taps(rng, 5, 1, 1, 2)
    L = [3, 3]
    ue_loop = oracle.OracleUE(L, 1, 1, [0, 1], taps, loop=True)
    ue_hold = oracle.OracleUE(L, 1, 1, [0, 1], taps, loop=False)
    for a in range(12):
        assert np.array_equal(oracle.anchor(ue_loop, a)[0, 0], taps[a % 5, 0, 0].astype(np.complex128))
        assert np.array_equal(oracle.anchor(ue_hold, a)[0, 0], taps[min(a, 4), 0, 0].astype(np.complex128))


# --------------------------------------------------------------------------
# 7. int16 packing: round half to even, saturation (numpy rint and clip)
# --------------------------------------------------------------------------
def test_packing_rounds_half_even_and_saturates():
    L = [4, 4]
    n = 8
    x = np.zeros((1, 4 * n, 2), dtype=np.int16)
    vals = np.array([1, 3, 5, -1, -3, 7, 9, -11, 20001, -20001, 32767, -32768] * 3)[: 4 * n]
    x[0, :, 0] = vals
    x[0, :, 1] = vals[::-1]
    for hval in (0.5, 1.5, 2.0):
        taps = np.full((9, 1, 1, 1), hval, dtype=np.complex64)
        ue = oracle.OracleUE(L, 1, 1, [0], taps)
        y, q = oracle.run_ue(ue, x)
        ref = np.clip(np.rint(iq_to_complex(x[0]).real * hval), -32768, 32767)
        assert np.array_equal(q[0, :, 0], ref.astype(np.int16))
        assert np.array_equal(y[0].real, iq_to_complex(x[0]).real * hval)


# --------------------------------------------------------------------------
# 8. AWGN: Gaussian law, variance, whiteness, independence, determinism
# --------------------------------------------------------------------------
def test_noise_statistics():
    from scipy import stats
    L = [139 * 16] + [137 * 16] * 13
    n = sum(L)
    var = 20971.52                         # SNR 20 dB at P_x = 2^21
    taps = np.zeros((15, 2, 1, 1), dtype=np.complex64)     # channel off: y = w
    ue = oracle.OracleUE(L, 1, 2, [0], taps, seed=0x77170002, ue_id=3, noise_var=var)
    x = np.zeros((1, n, 2), dtype=np.int16)
    y, _ = oracle.run_ue(ue, x, s_first=0)
    w0, w1 = y[0], y[1]
    m = len(w0)
    assert abs(np.mean(np.abs(w0) ** 2) / var - 1) < 0.02
    assert abs(np.mean(w0.real)) < 4 * np.sqrt(var / 2 / m)
    assert abs(np.var(w0.real) / np.var(w0.imag) - 1) < 0.03
    z = np.concatenate([w0.real, w0.imag]) / np.sqrt(var / 2)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    for lag in (1, 2, 3, 64):
        c = np.vdot(w0[:-lag], w0[lag:]) / np.vdot(w0, w0)
        assert abs(c) < 4 / np.sqrt(m)
    c01 = np.vdot(w0, w1) / np.sqrt(np.vdot(w0, w0).real * np.vdot(w1, w1).real)
    assert abs(c01) < 4 / np.sqrt(m)
    # re and im of one sample are uncorrelated
    assert abs(np.mean(w0.real * w0.imag)) / (var / 2) < 4 / np.sqrt(m)


def test_noise_keyed_by_absolute_sample_not_by_call():
    L = [5, 5]
    taps = np.zeros((40, 1, 1, 1), dtype=np.complex64)
    ue = oracle.OracleUE(L, 1, 1, [0], taps, seed=99, ue_id=5, noise_var=100.0)
    x = np.zeros((1, 6 * 10, 2), dtype=np.int16)
    y_all, _ = oracle.run_ue(ue, x, s_first=2)
    y_b, _ = oracle.run_ue(ue, x[:, 30:], s_first=5)
    assert np.array_equal(y_all[0, 30:], y_b[0])
    for i in (0, 7, 33):
        assert oracle.noise(99, 5, 0, 20 + i, 100.0) == y_all[0, i]
    other = oracle.OracleUE(L, 1, 1, [0], taps, seed=99, ue_id=6, noise_var=100.0)
    y_o, _ = oracle.run_ue(other, x, s_first=2)
    assert not np.any(y_o[0] == y_all[0])


def test_philox_statistics_and_avalanche():
    """Philox4x32-10 output words are uniform and every input bit avalanches."""
    key = (0x12345678, 0x9ABCDEF0)
    words = np.array([oracle.philox4x32_10((i, 0, 7, 1), key) for i in range(4096)], dtype=np.uint32)
    bits = np.unpackbits(words.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 4 * 0.5 / np.sqrt(bits.size)
    from scipy import stats
    counts = np.bincount(words.view(np.uint8).ravel(), minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-4
    base = oracle.philox4x32_10((5, 6, 7, 8), key)
    flips = []
    for word in range(4):
        for bit in (0, 13, 31):
            c = [5, 6, 7, 8]
            c[word] ^= 1 << bit
            o = oracle.philox4x32_10(c, key)
            flips.append(int(np.unpackbits((o ^ base).view(np.uint8)).sum()))
    for b in (0, 31):
        k2 = (key[0] ^ (1 << b), key[1])
        o = oracle.philox4x32_10((5, 6, 7, 8), k2)
        flips.append(int(np.unpackbits((o ^ base).view(np.uint8)).sum()))
    assert min(flips) > 35 and max(flips) < 93          # ~64 of 128 bits
    # distinct counters give distinct blocks (a bijection per key)
    assert len({tuple(w) for w in words}) == len(words)


# --------------------------------------------------------------------------
# 9. sparse top-n taps (Sec. III-C)
# --------------------------------------------------------------------------
def test_top_n_selects_dominant_taps():
    rng = np.random.default_rng(9)
    L = [6, 5, 5]
    n = sum(L)
    d = np.array([0, 2, 5, 9], dtype=np.int32)
    taps = _rand_taps(rng, 3 * 4 + 1, 1, 1, 4)
    x = rng.integers(-900, 900, size=(1, 3 * n, 2)).astype(np.int16)
    full, _ = oracle.run_ue(oracle.OracleUE(L, 1, 1, d, taps), x)
    same, _ = oracle.run_ue(oracle.OracleUE(L, 1, 1, d, taps, top_n=4), x)
    assert np.array_equal(full, same)
    # a static profile whose tap 2 dominates: top-1 keeps exactly that tap
    st = np.tile(np.array([0.1, 0.2j, 3 - 1j, 0.3], dtype=np.complex64).reshape(1, 1, 1, 4), (13, 1, 1, 1))
    y1, _ = oracle.run_ue(oracle.OracleUE(L, 1, 1, d, st, top_n=1), x)
    xc = iq_to_complex(x[0])
    ref = np.zeros_like(xc)
    ref[5:] = (3 - 1j) * xc[:-5]
    assert np.allclose(y1[0], ref, rtol=0, atol=1e-9)


TOPN_CASES = [
    # symbol_len, n_tx, n_rx, delays, n_slots, step_samples, top_n
    ([6, 5, 5], 1, 1, [0, 2, 5, 9, 11], 2, 0, 2),
    ([5, 4, 4, 4], 2, 2, [0, 1, 3, 7, 8, 20], 2, 0, 3),
    ([4, 4], 1, 2, [0, 3, 9, 10], 3, 5.5, 1),           # selection from trace-time anchors
]


@pytest.mark.parametrize("case", range(len(TOPN_CASES)))
def test_top_n_equals_exact_brute_force(case):
    """The per-symbol, per-link selection (Sec. III-C) and the convolution with only the kept taps
    agree with the exact rational brute force, which compares the powers exactly; the selection
    changes from symbol to symbol here (taps drawn per anchor)."""
    L, n_tx, n_rx, d, n_slots, step, top_n = TOPN_CASES[case]
    rng = np.random.default_rng(300 + case)
    n = sum(L)
    T = int(np.ceil(n_slots * n / step)) + 3 if step else len(L) * n_slots + 1
    taps = _rand_taps(rng, T, n_rx, n_tx, len(d))
    x = rng.integers(-3000, 3000, size=(n_tx, n_slots * n, 2)).astype(np.int16)
    ue = oracle.OracleUE(L, n_tx, n_rx, d, taps, step_samples=step, top_n=top_n)
    y, q = oracle.run_ue(ue, x)
    ye, qe = brute.run_exact(L, d, taps, x, step_samples=step, top_n=top_n)
    ye = brute.to_complex(ye)
    assert nrmse(y, ye) < 1e-13
    assert np.array_equal(q, qe)
    full, _ = oracle.run_ue(oracle.OracleUE(L, n_tx, n_rx, d, taps, step_samples=step), x)
    assert nrmse(y, full) > 1e-3                          # the sparse result really differs


def test_top_n_is_decided_on_fp64_powers():
    """Tap 1 = 1 + 2^-12 i has power 1 + 2^-24, above tap 0's power 1 by less than binary32 can
    resolve at 1.  The oracle ranks in FP64 and keeps tap 1, as the exact brute force does."""
    L = [4, 4]
    d = np.array([0, 2, 3], dtype=np.int32)
    prof = np.array([1.0, 1.0 + 2.0 ** -12 * 1j, 0.5], dtype=np.complex64)
    taps = np.tile(prof.reshape(1, 1, 1, 3), (3, 1, 1, 1))
    rng = np.random.default_rng(12)
    x = rng.integers(-2000, 2000, size=(1, 8, 2)).astype(np.int16)
    y, q = oracle.run_ue(oracle.OracleUE(L, 1, 1, d, taps, top_n=1), x)
    xc = iq_to_complex(x[0])
    ref = np.zeros_like(xc)
    ref[2:] = complex(prof[1]) * xc[:-2]
    assert np.allclose(y[0], ref, rtol=0, atol=1e-9)
    ye, qe = brute.run_exact(L, d, taps, x, top_n=1)
    assert nrmse(y, brute.to_complex(ye)) < 1e-13 and np.array_equal(q, qe)


def test_explicit_selection_replaces_the_top_n_rule():
    """An explicit tap mask: all taps kept gives the dense result; the FP64 selection of
    tests.helpers.topn_selections gives the top-n result; one kept tap of a static profile gives
    that tap's delayed copy of the input."""
    rng = np.random.default_rng(13)
    L = [5, 4, 4]
    n = sum(L)
    d = np.array([0, 1, 4, 6], dtype=np.int32)
    taps = _rand_taps(rng, 2 * 3 + 1, 2, 1, 4)
    x = rng.integers(-900, 900, size=(1, 2 * n, 2)).astype(np.int16)
    ue = oracle.OracleUE(L, 1, 2, d, taps, top_n=2)
    dense, _ = oracle.run_ue(oracle.OracleUE(L, 1, 2, d, taps), x)
    y_all, _ = oracle.run_ue(ue, x, keep=np.ones((7, 2, 1, 4), dtype=bool))
    assert np.array_equal(y_all, dense)
    base = np.stack([topn_selections(oracle.anchor(ue, a), 2)[0] for a in range(7)])
    assert base.sum(axis=-1).max() == 2 and base.sum(axis=-1).min() == 2
    y_sel, _ = oracle.run_ue(ue, x, keep=base)
    y_rule, _ = oracle.run_ue(ue, x)
    assert np.array_equal(y_sel, y_rule)
    st = np.tile(np.array([0.5, 2 - 1j, 0.25j, 1.0], dtype=np.complex64).reshape(1, 1, 1, 4), (7, 2, 1, 1))
    one = np.zeros((7, 2, 1, 4), dtype=bool)
    one[..., 2] = True                                    # keep only tap 2 (delay 4)
    y1, _ = oracle.run_ue(oracle.OracleUE(L, 1, 2, d, st, top_n=1), x, keep=one)
    xc = iq_to_complex(x[0])
    ref = np.zeros_like(xc)
    ref[4:] = 0.25j * xc[:-4]
    assert np.allclose(y1, np.stack([ref, ref]), rtol=0, atol=1e-9)


def test_topn_selections_lists_only_near_ties():
    """The valid-selection enumerator of the top-n GPU check: a clear ranking has one selection;
    powers within binary32 rounding of the n-th place allow each of the near-tied taps."""
    H = np.array([[[3.0, 1.0, 2.0, 0.5]]], dtype=np.complex128)
    base, alts = topn_selections(H, 2)
    assert base[0, 0].tolist() == [True, False, True, False] and not alts
    H = np.array([[[3.0, 1.0, 1.0 + 2.0 ** -30, 0.5, 1.0]]], dtype=np.complex128)
    base, alts = topn_selections(H, 2)
    assert base[0, 0].tolist() == [True, False, True, False, False]
    sels = [m.tolist() for m in alts[(0, 0)]]
    assert sels[0] == base[0, 0].tolist() and len(sels) == 3
    assert [True, True, False, False, False] in sels and [True, False, False, False, True] in sels
    base, alts = topn_selections(H, 0)
    assert base.all() and not alts


def test_top_n_ties_keep_the_lower_tap_and_follow_each_anchor():
    """Equal powers: the lower tap index wins.  A static profile whose dominant tap moves from
    index 1 (anchor 0) to index 3 (anchor 1) makes top-1 switch taps at the symbol boundary."""
    L = [4, 4]
    d = np.array([0, 1, 2, 3], dtype=np.int32)
    x = np.zeros((1, 8, 2), dtype=np.int16)
    x[0, 0, 0] = 1000                                     # unit impulse of height 1000 at sample 0
    # anchors: tap powers equal (1, 1j, -1, 0.5 - 0.5j has 0.5) -> top-1 keeps tap 0
    eq = np.array([1.0, 1j, -1.0, 0.5 - 0.5j], dtype=np.complex64).reshape(1, 1, 1, 4)
    y, _ = oracle.run_ue(oracle.OracleUE(L, 1, 1, d, np.tile(eq, (3, 1, 1, 1)), top_n=1), x)
    assert np.allclose(y[0, :4], [1000, 0, 0, 0], atol=1e-9)
    # anchor 0 favours tap 1, anchor 1 tap 3 (taps interpolate toward the next anchor)
    a0 = np.array([0.1, 2.0, 0.1, 0.1], dtype=np.complex64)
    a1 = np.array([0.1, 0.1, 0.1, 3.0], dtype=np.complex64)
    taps = np.stack([a0, a1, a1]).reshape(3, 1, 1, 4)
    x2 = np.zeros((1, 8, 2), dtype=np.int16)
    x2[0, :, 0] = 100                                     # constant input: y = sum of kept taps
    y2, _ = oracle.run_ue(oracle.OracleUE(L, 1, 1, d, taps, top_n=1), x2)
    for m in range(4):                                    # symbol 0 keeps tap 1 (delay 1)
        h = a0[1] + (m / 4) * (a1[1] - a0[1])
        assert abs(y2[0, m] - (100 * h if m >= 1 else 0)) < 1e-4
    for m in range(4, 8):                                 # symbol 1 keeps tap 3 (delay 3)
        assert abs(y2[0, m] - 100 * a1[3]) < 1e-4


# --------------------------------------------------------------------------
# 10. uplink aggregation at a cell (Sec. III-A: the gNB convolves and aggregates)
# --------------------------------------------------------------------------
def _cell_members(rng, n_members, L, n_rx, d, n_slots):
    n = sum(L)
    ues, xs = [], []
    for u in range(n_members):
        taps = _rand_taps(rng, len(L) * n_slots + 1, n_rx, 1, len(d))
        ues.append(oracle.OracleUE(L, 1, n_rx, d, taps, ue_id=u))
        xs.append(rng.integers(-2000, 2000, size=(1, n_slots * n, 2)).astype(np.int16))
    return ues, xs


def test_cell_of_one_member_is_that_member_with_the_cell_noise():
    """One member: the cell output is the member's own run with AWGN under the cell's key
    (same FP64 operations in the same order, so bit-identical)."""
    rng = np.random.default_rng(61)
    L, d = [6, 5, 5], [0, 2, 7]
    ues, xs = _cell_members(rng, 1, L, 2, d, 3)
    nv = 300.0
    yc, qc = oracle.run_cell(ues, xs, seed=0x1234, cell_id=9, noise_var=nv, s_first=2)
    u = ues[0]
    with_noise = oracle.OracleUE(L, 1, 2, d, u.taps, seed=0x1234, ue_id=9, noise_var=nv)
    y1, q1 = oracle.run_ue(with_noise, xs[0], s_first=2)
    assert np.array_equal(yc, y1) and np.array_equal(qc, q1)


def test_cell_sums_members_superposition():
    """Members with the same channel and inputs x1, x2 add up to one member fed x1 + x2 (the
    convolution is linear, so the aggregate is a sum, not an average or a selection); a member
    with zero input contributes nothing."""
    rng = np.random.default_rng(62)
    L, d = [8, 7, 7], [0, 1, 5, 12]
    n = sum(L)
    taps = _rand_taps(rng, 3 * 3 + 1, 1, 1, len(d))
    a = oracle.OracleUE(L, 1, 1, d, taps, ue_id=0)
    b = oracle.OracleUE(L, 1, 1, d, taps, ue_id=1)
    x1 = rng.integers(-9000, 9000, size=(1, 3 * n, 2)).astype(np.int16)
    x2 = rng.integers(-9000, 9000, size=(1, 3 * n, 2)).astype(np.int16)
    yc, _ = oracle.run_cell([a, b], [x1, x2], seed=1, cell_id=0)
    ysum, _ = oracle.run_ue(a, (x1.astype(np.int32) + x2).astype(np.int16))
    assert nrmse(yc, ysum) < 1e-13
    y0, _ = oracle.run_cell([a, b], [x1, np.zeros_like(x2)], seed=1, cell_id=0)
    ya, _ = oracle.run_ue(a, x1)
    assert np.array_equal(y0, ya)
    # three members, one of them silent, in any order give the same aggregate up to rounding
    ues, xs = _cell_members(rng, 3, L, 1, d, 3)
    xs[1] = np.zeros_like(xs[1])
    y012, _ = oracle.run_cell(ues, xs, seed=1, cell_id=0)
    y20, _ = oracle.run_cell([ues[2], ues[0]], [xs[2], xs[0]], seed=1, cell_id=0)
    assert nrmse(y012, y20) < 1e-14


# --------------------------------------------------------------------------
# 11. continuous CIR -> fixed delay grid (Sec. IV)
# --------------------------------------------------------------------------
def test_cir_resampling_closed_forms():
    """On-grid paths give exact impulses; a half-sample delay gives sinc(k - 1/2) =
    2 (-1)^(k+1) / (pi (2k - 1)); paths add linearly; a band-limited signal sampled on the grid
    is reproduced by summing its sinc-shifted copies (the interpolation identity)."""
    T, P, K = 3, 4, 12
    rng = np.random.default_rng(71)
    a = (rng.standard_normal((T, 2, 1, P)) + 1j * rng.standard_normal((T, 2, 1, P)))
    tau = np.tile(np.array([0.0, 3.0, 7.0, 11.0]), (T, 1))
    h = oracle.resample_cir(a, tau, K)
    ref = np.zeros((T, 2, 1, K), dtype=np.complex128)
    for p, d in enumerate([0, 3, 7, 11]):
        ref[..., d] += a[..., p]
    assert np.array_equal(h, ref)
    half = oracle.resample_cir(np.ones((1, 1, 1, 1)), np.array([[0.5]]), K)[0, 0, 0]
    k = np.arange(K)
    assert np.allclose(half, 2 * (-1.0) ** (k + 1) / (np.pi * (2 * k - 1)), rtol=0, atol=1e-15)
    tau2 = rng.uniform(0, K - 1, size=(T, P))
    h2 = oracle.resample_cir(a, tau2, K)
    parts = sum(oracle.resample_cir(a[..., p:p + 1], tau2[:, p:p + 1], K) for p in range(P))
    assert np.allclose(h2, parts, rtol=0, atol=1e-13)
    # interpolation identity: sum_p sinc(k - p) f(p) = f(k) for samples on the grid
    f = rng.standard_normal(K)
    ident = oracle.resample_cir(f.reshape(1, 1, 1, K), np.arange(K, dtype=float).reshape(1, K), K)
    assert np.allclose(ident[0, 0, 0], f, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------
# 12. sum-of-sinusoids tap processes (Sec. IV, Jakes-based Doppler)
# --------------------------------------------------------------------------
def test_sos_taps_have_unit_power_and_the_jakes_autocorrelation():
    """With the Zheng-Xiao parameters each process has E|h|^2 = amplitude^2 and the normalised
    autocorrelation of the classic Jakes spectrum, J0(2 pi f_D tau) (Bessel function of the first
    kind, order 0); a wrong frequency set, scale or 2 pi factor breaks one of them."""
    from scipy.special import j0
    from paper_2601_08217_gb300 import inputs
    rng = np.random.default_rng(91)
    f_d, m = 100.0, 16
    amp, freq, phase = inputs.sos_params(rng, f_d, np.full(400, 2.0), 4, 2, m)   # 3200 processes, power 1 each
    taus = np.array([0.0, 0.5e-3, 1e-3, 2e-3, 3.8e-3, 6e-3])
    t0 = rng.uniform(0.0, 10.0, size=8)
    acc = np.zeros(len(taus), dtype=np.complex128)
    pw = 0.0
    for t in t0:
        h = oracle.sos_taps(amp, freq, phase, t + taus)                          # [len(taus)][4][2][400]
        acc += (h * np.conj(h[0])[None]).reshape(len(taus), -1).mean(axis=1)
        pw += np.mean(np.abs(h[0]) ** 2)
    acc /= len(t0)
    assert abs(pw / len(t0) - 1.0) < 0.03
    assert np.allclose(acc.real, j0(2 * np.pi * f_d * taus), atol=0.04)
