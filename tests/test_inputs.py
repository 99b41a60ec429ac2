"""Checks of the seeded input generators (CPU only)."""
import os

import numpy as np
from scipy.special import j0

from paper_2601_08217_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "nr_30khz_symbol_lengths.txt")


def test_nr_symbol_lengths_match_38211_table():
    rows = [list(map(int, l.split())) for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for n_fft, first, other, slot in rows:
        L = inputs.nr_symbol_lengths(n_fft)
        assert L[0] == first and all(v == other for v in L[1:]) and sum(L) == slot and len(L) == 14


def test_iq_generator_is_seeded_int16_gaussian():
    a = inputs.gen_iq(inputs.rng_for(2, 3, 0), 1, 200000)
    b = inputs.gen_iq(inputs.rng_for(2, 3, 0), 1, 200000)
    assert a.dtype == np.int16 and np.array_equal(a, b)
    assert abs(a.astype(np.float64).std() / 1024.0 - 1) < 0.01


def test_delays_are_sorted_distinct_and_bounded():
    d = inputs.gen_delays(inputs.rng_for(2, 0, 0, 1), 24, 256)
    assert d[0] == 0 and np.all(np.diff(d) > 0) and d.max() <= 256 and len(d) == 24


def test_jakes_autocorrelation_follows_bessel_j0():
    rng = np.random.default_rng(11)
    f_d = 100.0
    t = np.arange(4000) * 1e-4
    g = inputs.jakes_sos(rng, t, f_d, 400)
    assert abs(np.mean(np.abs(g) ** 2) - 1) < 0.05
    for lag in (0, 5, 10, 20, 38):
        r = np.mean(g[lag:] * np.conj(g[: len(t) - lag])).real
        assert abs(r - j0(2 * np.pi * f_d * lag * 1e-4)) < 0.06


def test_trace_power_profile():
    spec = inputs.make_ue(2, 0, 2048, 24, 256, 100.0, 4)
    assert spec.taps.shape == (14 * 4 + 1, 1, 1, 24)
    assert spec.n == 30720
    p = inputs.pdp_span_decay(spec.delays)
    assert abs(p.sum() - 1) < 1e-12 and abs(p[0] / p[-1] - 100.0 ** (spec.delays[-1] / spec.delays.max())) < 1e-6
