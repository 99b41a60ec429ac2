"""Allocator hook: an engine whose device buffers come from PyTorch's caching allocator.

Bars: every kernel form (dense FP32, top-n, tensor-core BF16, an uplink cell) gives the same bits as
the same engine on cudaMalloc; the hook holds at least the engine's admitted bytes while channels
live; destroying a channel and then the engine hands every buffer back; a serving run (whose
thread may grow work lists through the hook) completes its requests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc

pytestmark = pytest.mark.gpu

N_SLOTS = 3


def _specs():
    dense = inputs.make_ue(21, 0, 1024, 16, 200, 100.0, N_SLOTS + 2, n_tx=2, n_rx=2, snr_db=20.0)
    sparse = inputs.make_ue(21, 1, 1024, 24, 300, 100.0, N_SLOTS + 2, snr_db=20.0)
    tcore = inputs.make_ue(21, 2, 1024, 32, 64, 100.0, N_SLOTS + 2, n_tx=2, n_rx=2)
    return [(dense, {}), (sparse, dict(top_n=6)), (tcore, dict(precision=tc.TT_BF16_TC, cf32=True))]


def _run(allocator):
    eng = tc.Engine(persistent=True, allocator=allocator)
    outs = []
    try:
        chans = []
        for sp, kw in _specs():
            chans.append(tc.Chan(eng, sp, ring_slots=N_SLOTS + 3, **kw))
        members = [inputs.make_ue(22, 10 + u, 1024, 12, 100, 100.0, N_SLOTS + 2) for u in range(2)]
        cell = tc.Cell(eng, cell_id=3, samples_per_slot=members[0].n, ring_slots=N_SLOTS + 1, noise_var=1.0)
        for sp in members:
            ch = tc.Chan(eng, sp, cf32=True, ring_slots=N_SLOTS + 3)
            cell.attach(ch)
            chans.append(ch)
        specs = [s for s, _ in _specs()] + members
        for ch, sp in zip(chans, specs):
            ch.push(0, inputs.make_iq(23, sp, N_SLOTS))
        eng.run()
        outs = [ch.pull(0, N_SLOTS) for ch in chans[:3]] + [cell.pull(0, N_SLOTS)]
        stats = eng.stats()
        held = allocator.live_bytes if allocator is not None else None
        if allocator is not None:
            before = allocator.live_bytes
            one = chans[0]
            one.destroy()
            assert allocator.live_bytes < before          # the channel's buffers went back
    finally:
        eng.close()
    return outs, stats, held


def test_engine_on_the_torch_caching_allocator():
    base, _, _ = _run(None)
    hook = tc.TorchAllocator(0)
    got, stats, held = _run(hook)
    for a, b in zip(base, got):
        assert np.array_equal(a, b)
    assert held >= stats["hbm_in_use"]
    assert hook.live == {}                               # every buffer returned at engine close
    torch.cuda.synchronize()


def test_serving_through_the_hook():
    hook = tc.TorchAllocator(0)
    eng = tc.Engine(persistent=True, allocator=hook)
    try:
        for u in range(4):
            sp = inputs.make_ue(24, u, 1024, 12, 100, 100.0, 6)
            tc.Chan(eng, sp, ring_slots=6, top_n=4 if u % 2 else 0)
        rep = tc.tt_engine_serve(eng.h, duration_s=0.1, warmup_s=0.01, slot_period_us=500.0, jitter_us=50.0,
                                 deadline_us=500.0, seed=5, release_outputs=True)
        assert rep["completed"] > 0.9 * rep["requests"] > 0
    finally:
        eng.close()
    assert hook.live == {}


def test_hooks_must_come_in_pairs():
    hook = tc.TorchAllocator(0)
    cfg = tc.EngineConfig(C.sizeof(tc.EngineConfig), 0, 0, tc.TT_FORM_BATCHED, 0, 0, 0, 0, 0)
    cfg.dev_alloc = hook.alloc_fn                        # dev_free left NULL
    h = C.c_void_p()
    assert tc.load().tt_engine_create(C.byref(cfg), C.byref(h)) == tc.TT_ERR_INVALID
    assert "together" in tc.tt_last_error()
