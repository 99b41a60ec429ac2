"""tt_conv_static: the entry point for callers that may not allocate device memory.

Such callers (code running inside another framework's memory pool, a
pre-sized real-time partition, anything that must keep a fixed footprint)
cannot use the engine, which allocates rings and work lists.  tt_conv_static
runs the same kernel on buffers the caller owns, with its scratch in a fixed
array inside the library.  This file is collected last so that a failure here
does not hide any other test.
"""
import numpy as np
import pytest
import torch

from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.gpu_harness import run_gpu

pytestmark = pytest.mark.gpu


def _specs():
    return [inputs.make_ue(2, 0, 2048, 24, 256, 100.0, 8, snr_db=20.0),
            inputs.make_ue(5, 1, 1024, 12, 300, 50.0, 8, n_tx=2, n_rx=2, snr_db=15.0)]


def _static_desc(spec, d_in, d_out, d_taps, q, first, n):
    return dict(symbol_len=spec.symbol_len, n_tx=spec.n_tx, n_rx=spec.n_rx, ring_slots=q, d_ring_in=d_in,
                d_ring_out=d_out, d_taps=d_taps, delays=spec.delays, n_anchors=spec.taps.shape[0],
                step_samples=spec.step_samples, loop=spec.loop, seed=spec.seed, noise_var=spec.noise_var,
                ue_id=spec.ue_id, first_slot=first, n_slots=n)


def test_static_entry_matches_engine_on_two_calls():
    tc.load()
    specs = _specs()
    n_slots, q = 6, 8
    xs = [inputs.make_iq(2 + i, sp, n_slots) for i, sp in enumerate(specs)]
    ref = run_gpu(specs, xs, n_slots, cf32=False)          # the engine path
    dev = []
    for sp, x in zip(specs, xs):
        d_in = torch.zeros((q, sp.n_tx, sp.n, 2), dtype=torch.int16, device="cuda")
        d_in[:n_slots] = torch.from_numpy(tc.slots_major(x, sp.n)).cuda()
        d_out = torch.zeros((q, sp.n_rx, sp.n, 2), dtype=torch.int16, device="cuda")
        d_taps = torch.from_numpy(np.ascontiguousarray(sp.taps).view(np.float32).copy()).cuda()
        dev.append((d_in, d_out, d_taps))
    stream = torch.cuda.current_stream()
    for first in (0, 3):                                     # two calls in a row
        tc.tt_conv_static([_static_desc(sp, *d, q, first, 3) for sp, d in zip(specs, dev)], stream)
    torch.cuda.synchronize()
    for sp, d, r in zip(specs, dev, ref):
        got = tc.antenna_major(d[1][:n_slots].cpu().numpy())
        assert np.abs(got.astype(np.int32) - r.astype(np.int32)).max() <= 1
    # a third call reuses the scratch array: no device memory is taken
    free0 = torch.cuda.mem_get_info()[0]
    tc.tt_conv_static([_static_desc(sp, *d, q, 0, 3) for sp, d in zip(specs, dev)], stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


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
