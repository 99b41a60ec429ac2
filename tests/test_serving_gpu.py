"""Serving form: Poisson slot requests from many UEs, continuous batching, latency report.

The results a UE gets while served in the mix equal the results of the same
UE run alone (bit for bit), and a full ring refuses requests instead of
corrupting state."""
import numpy as np
import pytest

from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.gpu_harness import hist_slots

pytestmark = pytest.mark.gpu

PREFILL = 8


def _prefill(eng, specs, ring_extra, n=PREFILL):
    chans = []
    for i, sp in enumerate(specs):
        ch = tc.Chan(eng, sp, ring_slots=hist_slots(sp) + ring_extra)
        ch.push(0, tc.slots_major(inputs.make_iq(5, sp, n), sp.n))
        chans.append(ch)
    eng.run()
    for ch in chans:
        ch.pull(0, n)
    return chans


def test_each_result_is_the_same_alone_and_in_the_mix():
    specs = inputs.workload_serving(n_ues=16, n_slots_trace=4)
    per_ue = 4
    eng = tc.Engine(persistent=True)
    chans = _prefill(eng, specs, PREFILL + 2)
    rep = tc.tt_engine_serve(eng.h, duration_s=0.05, slot_period_us=500.0, jitter_us=50.0, seed=3,
                             max_slots_per_ue=per_ue, release_outputs=False)
    assert rep["requests"] == rep["completed"] == 16 * per_ue and rep["refused"] == 0
    assert rep["p50_us"] > 0 and rep["p99_us"] >= rep["p50_us"] and rep["batches"] >= 1
    served = [ch.pull(PREFILL, per_ue) for ch in chans]
    eng.close()
    for i, sp in enumerate(specs):
        e1 = tc.Engine(persistent=False)
        (ch,) = _prefill(e1, [sp], PREFILL + 2)
        tc.tt_chan_commit_slots(ch.h, PREFILL, per_ue)     # the same ring positions, in place
        e1.run()
        alone = ch.pull(PREFILL, per_ue)
        e1.close()
        assert np.array_equal(alone, served[i]), i


def test_full_ring_refuses_requests():
    specs = inputs.workload_serving(n_ues=4, n_slots_trace=2)
    eng = tc.Engine()
    _prefill(eng, specs, 3, n=2)
    rep = tc.tt_engine_serve(eng.h, duration_s=0.02, slot_period_us=200.0, jitter_us=0.0, seed=1,
                             release_outputs=False)
    assert rep["refused"] > 0 and rep["completed"] == rep["requests"] - rep["refused"]
    eng.close()
