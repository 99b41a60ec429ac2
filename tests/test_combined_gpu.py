"""The widened features together, through the C ABI, against the oracle: a cell whose members are
a synthesised channel, a sparse (top-n) channel and a stored-trace channel; checkpoint/resume of
synthesised and sparse channels."""
import numpy as np
import pytest

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.helpers import nrmse
from tests.test_parity_gpu import Spec, assert_int16_close

pytestmark = pytest.mark.gpu

L = inputs.nr_symbol_lengths(1024)
FS = 30.72e6


def _sos_trace(amp, freq, phase, n_slots):
    n, nsym = sum(L), len(L)
    starts = np.concatenate([[0], np.cumsum(L)[:-1]])
    a = np.arange(n_slots * nsym + 1)
    b = (a // nsym) * n + starts[a % nsym]
    return oracle.sos_taps(amp, freq, phase, b / FS).astype(np.complex64)


def test_cell_of_synthesised_sparse_and_trace_members():
    rng = np.random.default_rng(131)
    ns, K = 3, 12
    d = inputs.gen_delays(rng, K, 150)
    amp, freq, phase = inputs.sos_params(rng, 200.0, inputs.pdp_span_decay(d, 20.0), 1, 1)
    synth_taps = _sos_trace(amp, freq, phase, ns)
    specs = [Spec(L, 1, 1, d, synth_taps),                                           # synthesised
             Spec(L, 1, 1, d, inputs.gen_trace(rng, np.arange(ns * 14 + 1) * 36e-6, 100.0,
                                                inputs.pdp_span_decay(d, 20.0), 1, 1)),  # sparse
             Spec(L, 1, 1, d, inputs.gen_trace(rng, np.arange(ns * 14 + 1) * 36e-6, 50.0,
                                                inputs.pdp_span_decay(d, 20.0), 1, 1))]  # trace
    xs = [np.clip(np.rint(rng.standard_normal((1, ns * sum(L), 2)) * 1024), -32768, 32767).astype(np.int16)
          for _ in specs]
    nv = inputs.noise_var_for_snr(25.0)
    ues = [oracle.OracleUE.from_spec(specs[0]), oracle.OracleUE.from_spec(specs[1], top_n=4),
           oracle.OracleUE.from_spec(specs[2])]
    y_ref, q_ref = oracle.run_cell(ues, xs, seed=77, cell_id=2, noise_var=nv)
    for cf32 in (True, False):
        eng = tc.Engine(persistent=True)
        try:
            cell = tc.Cell(eng, cell_id=2, samples_per_slot=sum(L), seed=77, noise_var=nv, ring_slots=ns, cf32=cf32)
            a = tc.Chan(eng, specs[0], load=False, cf32=True, ring_slots=ns + 2)
            tc.tt_chan_load_jakes(a.h, d, amp, freq, phase, FS)
            b = tc.Chan(eng, specs[1], cf32=True, ring_slots=ns + 2, top_n=4)
            c = tc.Chan(eng, specs[2], cf32=True, ring_slots=ns + 2)
            for ch in (a, b, c):
                cell.attach(ch)
            for ch, x in zip((a, b, c), xs):
                ch.push(0, x)
            eng.run()
            y = tc.antenna_major(cell.pull(0, ns))
        finally:
            eng.close()
        if cf32:
            assert nrmse(y, y_ref) <= 1e-5
        else:
            assert_int16_close(y, y_ref, q_ref)


@pytest.mark.parametrize("mode", ["synth", "sparse"])
def test_checkpoint_resume_of_synthesised_and_sparse_channels(mode):
    rng = np.random.default_rng(137)
    ns, K = 8, 10
    d = inputs.gen_delays(rng, K, 120)
    amp, freq, phase = inputs.sos_params(rng, 150.0, inputs.pdp_span_decay(d, 20.0), 1, 1)
    spec = Spec(L, 1, 1, d, _sos_trace(amp, freq, phase, ns), noise_var=inputs.noise_var_for_snr(20.0), seed=9)
    x = np.clip(np.rint(rng.standard_normal((1, ns * sum(L), 2)) * 1024), -32768, 32767).astype(np.int16)
    xs = tc.slots_major(x, sum(L))
    top = 3 if mode == "sparse" else 0

    def chan(eng):
        if mode == "synth":
            ch = tc.Chan(eng, spec, load=False, ring_slots=6)
            tc.tt_chan_load_jakes(ch.h, d, amp, freq, phase, FS)
            return ch
        return tc.Chan(eng, spec, ring_slots=6, top_n=top)

    eng = tc.Engine()
    try:
        ch = chan(eng)
        ch.push(0, xs[:4])
        eng.run()
        first = ch.pull(0, 4)
        eng.sync()
        blob = tc.tt_chan_get_state(ch.h)
    finally:
        eng.close()
    eng2 = tc.Engine()
    try:
        ch2 = chan(eng2)
        tc.tt_chan_set_state(ch2.h, blob)
        ch2.push(4, xs[4:])
        eng2.run()
        second = ch2.pull(4, 4)
    finally:
        eng2.close()
    resumed = tc.antenna_major(np.concatenate([first, second], axis=0))
    y_ref, q_ref = oracle.run_ue(oracle.OracleUE.from_spec(spec, top_n=top), x)
    assert_int16_close(resumed, y_ref, q_ref)
