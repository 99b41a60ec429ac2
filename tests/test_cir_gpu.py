"""Trace ingestion from a continuous CIR (Sec. IV: resampled onto the fixed delay grid per time
step) on the GPU, through the C ABI: the device-resampled trace drives the convolution, checked
against the oracle convolving with the oracle's own resampling."""
import numpy as np
import pytest

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.helpers import nrmse
from tests.test_parity_gpu import Spec, assert_int16_close

pytestmark = pytest.mark.gpu


def _cir(rng, T, n_rx, n_tx, P, max_tau, on_grid=False):
    g = (rng.standard_normal((T, n_rx, n_tx, P)) + 1j * rng.standard_normal((T, n_rx, n_tx, P))) / np.sqrt(2 * P)
    tau = rng.integers(0, int(max_tau), size=(T, P)).astype(np.float64) if on_grid else \
        rng.uniform(0.0, max_tau, size=(T, P))
    return g.astype(np.complex64), tau


def _run(spec, x, n_slots, gains, tau, K, cf32):
    eng = tc.Engine(persistent=True)
    try:
        ch = tc.Chan(eng, spec, load=False, cf32=cf32, ring_slots=n_slots + 2)
        tc.tt_chan_load_cir(ch.h, gains, tau, K, spec.step_samples, spec.loop)
        ch.push(0, x)
        eng.run()
        return tc.antenna_major(ch.pull(0, n_slots))
    finally:
        eng.close()


@pytest.mark.parametrize("n_rx,n_tx,step", [(1, 1, 0.0), (2, 2, 0.0), (1, 2, 30720.0)])
def test_cir_resampled_on_device_matches_oracle(n_rx, n_tx, step):
    rng = np.random.default_rng(81 + n_rx + 3 * n_tx)
    L = inputs.nr_symbol_lengths(1024)
    n, ns, K, P = sum(L), 3, 40, 6
    T = len(L) * ns + 1 if not step else int(np.ceil(ns * n / step)) + 2
    gains, tau = _cir(rng, T, n_rx, n_tx, P, K - 6)
    taps = oracle.resample_cir(gains, tau, K).astype(np.complex64)      # the trace, rounded like the device's
    spec = Spec(L, n_tx, n_rx, np.arange(K), taps, step=step, noise_var=inputs.noise_var_for_snr(25.0), seed=5)
    x = np.clip(np.rint(rng.standard_normal((n_tx, ns * n, 2)) * 1024), -32768, 32767).astype(np.int16)
    y_ref, q_ref = oracle.run_ue(oracle.OracleUE.from_spec(spec), x)
    y = _run(spec, x, ns, gains, tau, K, cf32=True)
    assert nrmse(y, y_ref) <= 1e-5
    q = _run(spec, x, ns, gains, tau, K, cf32=False)
    assert_int16_close(q, y_ref, q_ref)


def test_on_grid_cir_equals_the_tap_trace():
    """Paths on integer delays resample to exact impulses: the output equals that of the
    equivalent tap trace bit for bit."""
    rng = np.random.default_rng(88)
    L = [64, 64, 64, 64]
    n, ns, K, P = sum(L), 2, 32, 4
    T = len(L) * ns + 1
    gains, tau = _cir(rng, T, 1, 1, P, K, on_grid=True)
    taps = np.zeros((T, 1, 1, K), dtype=np.complex64)
    for t in range(T):
        for p in range(P):
            taps[t, 0, 0, int(tau[t, p])] += gains[t, 0, 0, p]
    spec = Spec(L, 1, 1, np.arange(K), taps)
    x = rng.integers(-3000, 3000, size=(1, ns * n, 2)).astype(np.int16)
    eng = tc.Engine()
    try:
        a = tc.Chan(eng, spec, ring_slots=ns + 2)
        a.push(0, x)
        eng.run()
        ref = a.pull(0, ns)
    finally:
        eng.close()
    got = _run(spec, x, ns, gains, tau, K, cf32=False)
    assert np.array_equal(got, tc.antenna_major(ref))


def test_cir_errors():
    spec = Spec([8, 8], 1, 1, [0, 1, 2, 3], np.ones((3, 1, 1, 4), dtype=np.complex64))   # max_taps 4
    eng = tc.Engine()
    try:
        ch = tc.Chan(eng, spec, load=False)
        g = np.ones((2, 1, 1, 2), dtype=np.complex64)
        for tau, K, status in ((np.array([[0.0, -1.0]] * 2), 4, tc.TT_ERR_TRACE),
                               (np.array([[0.0, np.nan]] * 2), 4, tc.TT_ERR_TRACE),
                               (np.array([[0.0, 1.5]] * 2), 40, tc.TT_ERR_TRACE)):
            with pytest.raises(tc.TTError) as ex:
                tc.tt_chan_load_cir(ch.h, g, tau, K)
            assert ex.value.status == status
    finally:
        eng.close()
