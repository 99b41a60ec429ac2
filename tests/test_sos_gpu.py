"""Sum-of-sinusoids tap processes synthesised on the device (Sec. IV: 3GPP traces with a
Jakes-based Doppler model), through the C ABI, against the oracle convolving with its own FP64
synthesis of the same anchors."""
import numpy as np
import pytest

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.helpers import nrmse
from tests.test_parity_gpu import Spec, assert_int16_close

pytestmark = pytest.mark.gpu


def _model(rng, n_rx, n_tx, K, f_d=300.0):
    d = inputs.gen_delays(rng, K, 200)
    pdp = inputs.pdp_span_decay(d, 20.0) if hasattr(inputs, "pdp_span_decay") else np.full(K, 1.0 / K)
    amp, freq, phase = inputs.sos_params(rng, f_d, pdp, n_rx, n_tx)
    return d, amp, freq, phase


def _oracle_taps(L, fs, s0, n_slots, amp, freq, phase):
    """Anchors of slots [s0, s0 + n_slots) plus the next one, at their absolute times."""
    n, nsym = sum(L), len(L)
    starts = np.concatenate([[0], np.cumsum(L)[:-1]])
    a = np.arange(s0 * nsym, (s0 + n_slots) * nsym + 1)
    b = (a // nsym) * n + starts[a % nsym]
    return oracle.sos_taps(amp, freq, phase, b / fs).astype(np.complex64)


def _gpu(L, n_rx, n_tx, d, amp, freq, phase, fs, x, s0, n_slots, cf32, stream=False, prec=tc.TT_FP32):
    spec = Spec(L, n_tx, n_rx, d, np.zeros((1, n_rx, n_tx, len(d)), np.complex64))
    eng = tc.Engine(persistent=True)
    try:
        ch = tc.Chan(eng, spec, load=False, cf32=cf32, ring_slots=(3 if stream else n_slots + 2), precision=prec)
        tc.tt_chan_load_jakes(ch.h, d, amp, freq, phase, fs)
        if stream:
            outs = []
            for s in range(n_slots):
                ch.push(s0 + s, tc.slots_major(x, ch.n)[s:s + 1])
                eng.run()
                outs.append(ch.pull(s0 + s, 1))
            return tc.antenna_major(np.concatenate(outs, axis=0))
        ch.push(s0, x)
        eng.run()
        return tc.antenna_major(ch.pull(s0, n_slots))
    finally:
        eng.close()


@pytest.mark.parametrize("n_rx,n_tx,s0", [(1, 1, 0), (2, 2, 3), (1, 1, 200000)])
def test_synthesised_taps_match_oracle(n_rx, n_tx, s0):
    """s0 = 200000 puts the replay 100 s in: the FP64 phase reduction keeps the taps exact."""
    rng = np.random.default_rng(101 + n_rx + s0 % 7)
    L = inputs.nr_symbol_lengths(1024)
    fs, ns = 30.72e6, 3
    d, amp, freq, phase = _model(rng, n_rx, n_tx, 12)
    taps = _oracle_taps(L, fs, s0, ns, amp, freq, phase)
    spec = Spec(L, n_tx, n_rx, d, taps)                 # anchor 0 of this trace = slot s0's first symbol
    x = np.clip(np.rint(rng.standard_normal((n_tx, ns * sum(L), 2)) * 1024), -32768, 32767).astype(np.int16)
    y_ref, q_ref = oracle.run_ue(oracle.OracleUE.from_spec(spec), x)
    y = _gpu(L, n_rx, n_tx, d, amp, freq, phase, fs, x, s0, ns, cf32=True)
    assert nrmse(y, y_ref) <= 1e-5
    q = _gpu(L, n_rx, n_tx, d, amp, freq, phase, fs, x, s0, ns, cf32=False)
    assert_int16_close(q, y_ref, q_ref)


def test_synthesised_channel_streams_through_a_small_ring():
    """Slot by slot through a 3-slot ring the anchor ring wraps many times; the result equals the
    bulk run bit for bit."""
    rng = np.random.default_rng(109)
    L = [128] * 14
    d, amp, freq, phase = _model(rng, 1, 1, 8, f_d=500.0)
    ns = 12
    x = rng.integers(-2000, 2000, size=(1, ns * sum(L), 2)).astype(np.int16)
    bulk = _gpu(L, 1, 1, d, amp, freq, phase, 3.84e6, x, 5, ns, cf32=False)
    streamed = _gpu(L, 1, 1, d, amp, freq, phase, 3.84e6, x, 5, ns, cf32=False, stream=True)
    assert np.array_equal(bulk, streamed)


def test_synthesised_taps_drive_the_tensor_core_form():
    rng = np.random.default_rng(113)
    L = inputs.nr_symbol_lengths(1024)
    d = np.arange(32, dtype=np.int32)
    amp, freq, phase = inputs.sos_params(rng, 100.0, np.full(32, 1.0 / 32), 2, 2)
    fs, ns = 30.72e6, 1
    taps = _oracle_taps(L, fs, 0, ns, amp, freq, phase)
    spec = Spec(L, 2, 2, d, taps)
    x = np.clip(np.rint(rng.standard_normal((2, ns * sum(L), 2)) * 1024), -32768, 32767).astype(np.int16)
    y_ref, _ = oracle.run_ue(oracle.OracleUE.from_spec(spec), x)
    y = _gpu(L, 2, 2, d, amp, freq, phase, fs, x, 0, ns, cf32=True, prec=tc.TT_BF16_TC)
    assert 20 * np.log10(np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref)) < -40.0
