"""tt_conv_static: the entry point for callers that may not allocate device memory.

Such callers (code running inside another framework's memory pool, a
pre-sized real-time partition, anything that must keep a fixed footprint)
cannot use the engine, which allocates rings and work lists.  tt_conv_static
runs the same kernel on buffers the caller owns, with its scratch in a fixed
array inside the library.  It picks the engine's default samples per thread,
so its output must equal the engine's bit for bit; it is also held to the
oracle's bars.  This file is collected last so that a failure here does not
hide any other test.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.gpu_harness import hist_slots, run_gpu
from tests.helpers import nrmse
from tests.test_parity_gpu import Spec, assert_int16_close

pytestmark = pytest.mark.gpu

NRMSE_MAX = 1e-5


def _specs():
    return [inputs.make_ue(2, 0, 2048, 24, 256, 100.0, 8, snr_db=20.0),
            inputs.make_ue(5, 1, 1024, 12, 300, 50.0, 8, n_tx=2, n_rx=2, snr_db=15.0)]


def _static_desc(spec, d_in, d_out, d_taps, q, first, n, cf32=False):
    return dict(symbol_len=spec.symbol_len, n_tx=spec.n_tx, n_rx=spec.n_rx, ring_slots=q, d_ring_in=d_in,
                d_ring_out=d_out, d_taps=d_taps, delays=spec.delays, n_anchors=spec.taps.shape[0],
                step_samples=spec.step_samples, loop=spec.loop, seed=spec.seed, noise_var=spec.noise_var,
                ue_id=spec.ue_id, first_slot=first, n_slots=n,
                output_format=tc.TT_OUT_CF32 if cf32 else tc.TT_OUT_INT16)


def _device_rings(spec, x, n_slots, q, cf32=False):
    d_in = torch.zeros((q, spec.n_tx, spec.n, 2), dtype=torch.int16, device="cuda")
    d_in[:n_slots] = torch.from_numpy(tc.slots_major(x, spec.n)).cuda()
    if cf32:
        d_out = torch.zeros((q, spec.n_rx, spec.n, 2), dtype=torch.float32, device="cuda")
    else:
        d_out = torch.zeros((q, spec.n_rx, spec.n, 2), dtype=torch.int16, device="cuda")
    d_taps = torch.from_numpy(np.ascontiguousarray(spec.taps).view(np.float32).copy()).cuda()
    return d_in, d_out, d_taps


def _static_output(d_out, n_slots, cf32):
    o = d_out[:n_slots].cpu().numpy()
    if cf32:
        return tc.antenna_major(o[..., 0] + 1j * o[..., 1])
    return tc.antenna_major(o)


def test_static_entry_matches_engine_and_oracle_on_two_calls():
    tc.load()
    specs = _specs()
    n_slots, q = 6, 8
    xs = [inputs.make_iq(2 + i, sp, n_slots) for i, sp in enumerate(specs)]
    ref = run_gpu(specs, xs, n_slots, cf32=False)          # the engine path
    dev = [_device_rings(sp, x, n_slots, q) for sp, x in zip(specs, xs)]
    stream = torch.cuda.current_stream()
    for first in (0, 3):                                     # two calls in a row
        tc.tt_conv_static([_static_desc(sp, *d, q, first, 3) for sp, d in zip(specs, dev)], stream)
    torch.cuda.synchronize()
    for sp, x, d, r in zip(specs, xs, dev, ref):
        got = _static_output(d[1], n_slots, cf32=False)
        assert np.array_equal(got, r)                      # same kernel, same variant: bit for bit
        y_ref, q_ref = oracle.run_ue(oracle.OracleUE.from_spec(sp), x)
        assert_int16_close(got, y_ref, q_ref)
    # a third call reuses the scratch array: no device memory is taken
    free0 = torch.cuda.mem_get_info()[0]
    tc.tt_conv_static([_static_desc(sp, *d, q, 0, 3) for sp, d in zip(specs, dev)], stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_entry_timed_trace_looping_complex64():
    """A 1 ms trace (entries every 30720 samples at 20 MHz, FP64 trace time) that loops, with
    complex64 output, on two calls in a row, against the engine (bit for bit) and the oracle."""
    tc.load()
    sp = inputs.make_ue(6, 2, 1024, 10, 200, 300.0, 2, n_tx=1, n_rx=2, snr_db=25.0,
                        step_samples=30720.0, loop=True)
    n_slots = 6                                              # beyond the 2-slot trace: it wraps
    q = n_slots + hist_slots(sp)
    x = inputs.make_iq(6, sp, n_slots)
    ref = run_gpu([sp], [x], n_slots, cf32=True)[0]
    d = _device_rings(sp, x, n_slots, q, cf32=True)
    stream = torch.cuda.current_stream()
    for first in (0, 4):
        tc.tt_conv_static([_static_desc(sp, *d, q, first, 4 if first == 0 else 2, cf32=True)], stream)
    torch.cuda.synchronize()
    got = _static_output(d[1], n_slots, cf32=True)
    assert np.array_equal(got, ref)
    y_ref, _ = oracle.run_ue(oracle.OracleUE.from_spec(sp), x)
    assert nrmse(got, y_ref) <= NRMSE_MAX


def test_static_entry_at_the_minimum_ring_depth():
    """ring_slots = n_slots + history: the call's last slot takes the ring position just after the
    delay line of its first slot, which must still read zeros (the slots before the first)."""
    tc.load()
    rng = np.random.default_rng(8)
    n_slots = 5
    L = [64, 64, 64, 64]
    d = [0, 5, 130, 300, 600]                                 # the delay line spans 3 slots of 256
    z = rng.standard_normal((4 * n_slots + 1, 1, 1, len(d))) + 1j * rng.standard_normal((4 * n_slots + 1, 1, 1, len(d)))
    sp = Spec(L, 1, 1, d, (z / np.sqrt(2 * len(d))).astype(np.complex64), noise_var=300.0, seed=99, ue_id=4)
    h = hist_slots(sp)
    assert h == 3
    q = n_slots + h
    x = np.clip(np.rint(rng.standard_normal((1, n_slots * sp.n, 2)) * 1024), -32768, 32767).astype(np.int16)
    ref = run_gpu([sp], [x], n_slots)[0]
    d = _device_rings(sp, x, n_slots, q)
    tc.tt_conv_static([_static_desc(sp, *d, q, 0, n_slots)], torch.cuda.current_stream())
    torch.cuda.synchronize()
    got = _static_output(d[1], n_slots, cf32=False)
    assert np.array_equal(got, ref)
    y_ref, q_ref = oracle.run_ue(oracle.OracleUE.from_spec(sp), x)
    assert_int16_close(got, y_ref, q_ref)


def test_static_entry_rejects_sizes_beyond_its_limits():
    tc.load()
    sp = _specs()[0]
    d = torch.zeros(16, dtype=torch.int16, device="cuda")
    one = _static_desc(sp, d, d, d, 8, 0, 1)
    with pytest.raises(tc.TTError) as ei:
        tc.tt_conv_static([one] * 65)
    assert ei.value.status == tc.TT_ERR_INVALID and "at most 64" in str(ei.value)
    big = dict(one, symbol_len=[70000])
    with pytest.raises(tc.TTError) as ei:
        tc.tt_conv_static([big])
    assert ei.value.status == tc.TT_ERR_INVALID
