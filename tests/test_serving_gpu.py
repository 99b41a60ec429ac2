"""Serving form: Poisson slot requests from many UEs, continuous batching, latency report.

tt_engine_serve generates the arrivals and commits them through the engine's request path (the
batching thread of tt_server_start).  The results a UE gets while served in the mix equal the
results of the same UE run alone (bit for bit).  Arrivals that find a UE's ring full wait in a
bounded per-UE queue; only when that queue overflows is a request refused, and state is never
corrupted."""
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


def test_arrivals_beyond_a_full_ring_and_its_queue_are_refused():
    """Nothing pulls and outputs are kept, so each ring fills: the next 64 arrivals of a UE queue,
    later ones are refused, and every queued one still waiting at the end counts as refused."""
    specs = inputs.workload_serving(n_ues=4, n_slots_trace=2)
    eng = tc.Engine()
    _prefill(eng, specs, 3, n=2)
    rep = tc.tt_engine_serve(eng.h, duration_s=0.02, slot_period_us=200.0, jitter_us=0.0, seed=1,
                             release_outputs=False)
    assert rep["refused"] > 0 and rep["completed"] == rep["requests"] - rep["refused"]
    eng.close()


def test_sampled_ues_of_the_512ue_workload_match_the_oracle():
    """The 512-UE serving workload (20/40/100 MHz, SISO and 2x2, 6-48 taps, AWGN) served for a short
    run of 6 slots per UE.  32 UEs, every 16th, are checked over all their served slots against the
    oracle and against the same UE run alone.

    The serve loop replays each ring in place, so slot s reads ring position s mod Q.  Each sampled
    UE's ring is first filled at every position with its own IQ and released, so served slot s reads
    x[s mod Q], and the oracle runs on exactly that sequence."""
    import oracle
    from tests.helpers import nrmse
    from tests.test_parity_gpu import assert_int16_close
    specs = inputs.workload_serving(n_ues=512, n_slots_trace=4)
    per_ue, extra = 6, 10
    sampled = list(range(0, 512, 16))
    eng = tc.Engine(persistent=True)
    chans, qs, xs, parts = [], {}, {}, []
    for i, sp in enumerate(specs):
        q = hist_slots(sp) + extra
        ch = tc.Chan(eng, sp, ring_slots=q)
        n_fill = q if i in sampled else 2
        x = tc.slots_major(inputs.make_iq(5, sp, n_fill), sp.n)
        if i in sampled:
            qs[i], xs[i] = q, x
        # a push may fill the ring up to its history slots: the last ones go in a second round
        first = min(n_fill, q - hist_slots(sp))
        parts.append((x[:first], x[first:]))
        chans.append(ch)
    for rnd in range(2):
        s0 = [0 if rnd == 0 else len(p[0]) for p in parts]
        for ch, p, s in zip(chans, parts, s0):
            if len(p[rnd]):
                ch.push(s, p[rnd])
        eng.run()
        for ch, p, s in zip(chans, parts, s0):
            if len(p[rnd]):
                ch.pull(s, len(p[rnd]))
    rep = tc.tt_engine_serve(eng.h, duration_s=0.05, slot_period_us=500.0, jitter_us=50.0, seed=7,
                             max_slots_per_ue=per_ue, release_outputs=False)
    assert rep["requests"] == rep["completed"] == 512 * per_ue and rep["refused"] == 0
    served = {i: chans[i].pull(qs[i], per_ue) for i in sampled}
    eng.close()
    for i in sampled:
        sp, q, xsm = specs[i], qs[i], xs[i]
        n = sp.n
        # the input sequence the ring gives slots 0 .. q + per_ue - 1 ([n_tx][slots * N][2])
        seq = tc.antenna_major(xsm[[s % q for s in range(q + per_ue)]])
        y_ref, q_ref = oracle.run_ue(oracle.OracleUE.from_spec(sp), seq)
        got = tc.antenna_major(served[i])
        assert_int16_close(got, y_ref[:, q * n:], q_ref[:, q * n:])
        assert nrmse(got[..., 0] + 1j * got[..., 1], y_ref[:, q * n:]) < 1e-3   # int16 rounding only
        # alone: a fresh engine, the same ring contents, the same slots launched in place
        e1 = tc.Engine(persistent=False)
        c1 = tc.Chan(e1, sp, ring_slots=q)
        k = q - hist_slots(sp)
        for s0, blk in ((0, xsm[:k]), (k, xsm[k:])):
            c1.push(s0, blk)
            e1.run()
            c1.pull(s0, len(blk))
        tc.tt_chan_commit_slots(c1.h, q, per_ue)
        e1.run()
        alone = c1.pull(q, per_ue)
        e1.close()
        assert np.array_equal(alone, served[i]), i
