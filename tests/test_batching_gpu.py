"""Batching form: CUDA-graph replay with device-resident slot cursors, and the autotuner.

Each output sample is accumulated in the same order whatever the kernel
geometry, so graph replay, direct launches and every samples-per-thread
choice must agree bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.gpu_harness import hist_slots, run_gpu
from tests.helpers import nrmse

pytestmark = pytest.mark.gpu


def _stream(specs, xs, n_slots, engine_kw, per_run=1, autotune=False):
    eng = tc.Engine(**engine_kw)
    chans = [tc.Chan(eng, sp, ring_slots=hist_slots(sp) + 3 * per_run + 1) for sp in specs]
    if autotune:
        assert eng.autotune(reps=2) >= 0
    outs = [[] for _ in specs]
    s = 0
    while s < n_slots:
        k = min(per_run, n_slots - s)
        for ch, x in zip(chans, xs):
            ch.push(s, tc.slots_major(x, ch.n)[s:s + k])
        eng.run()
        for i, ch in enumerate(chans):
            outs[i].append(ch.pull(s, k))
        s += k
    st = eng.stats()
    eng.close()
    return [tc.antenna_major(np.concatenate(o, 0)) for o in outs], st


def test_graph_replay_equals_direct_launches():
    specs = inputs.workload_batching(n_ues=10, n_slots_trace=2)
    xs = [inputs.make_iq(3, sp, 6) for sp in specs]
    direct, _ = _stream(specs, xs, 6, dict(persistent=True))
    graph, st = _stream(specs, xs, 6, dict(persistent=True, graphs=True))
    for a, b in zip(direct, graph):
        assert np.array_equal(a, b)
    assert st["graph_builds"] == 1 and st["graph_launches"] == 6
    # a second shape (2 slots per run) rebuilds the graph once and stays correct
    graph2, st2 = _stream(specs, xs, 6, dict(persistent=True, graphs=True), per_run=2)
    for a, b in zip(direct, graph2):
        assert np.array_equal(a, b)
    assert st2["graph_builds"] == 1 and st2["graph_launches"] == 3


def test_graph_replay_against_oracle_and_after_resume():
    spec = inputs.make_ue(3, 4, 2048, 20, 400, 300.0, 8, snr_db=20.0, loop=True)
    x = inputs.make_iq(3, spec, 8)
    y_ref, q_ref = oracle.run_ue(oracle.OracleUE.from_spec(spec), x)
    eng = tc.Engine(graphs=True, persistent=True)
    ch = tc.Chan(eng, spec, ring_slots=4)
    xs = tc.slots_major(x, spec.n)
    got = []
    for s in range(4):
        ch.push(s, xs[s:s + 1])
        eng.run()
        got.append(ch.pull(s, 1))
    eng.sync()
    blob = tc.tt_chan_get_state(ch.h)
    ch.destroy()
    ch2 = tc.Chan(eng, spec, ring_slots=4)        # same engine: the cached graph's cursor is stale
    tc.tt_chan_set_state(ch2.h, blob)
    for s in range(4, 8):
        ch2.push(s, xs[s:s + 1])
        eng.run()
        got.append(ch2.pull(s, 1))
    eng.close()
    q = tc.antenna_major(np.concatenate(got, 0))
    d = np.abs(q.astype(np.int32) - q_ref.astype(np.int32))
    assert d.max() <= 1 and np.count_nonzero(d) < 1e-4 * d.size


def test_autotuner_keeps_results_bit_identical():
    specs = inputs.workload_batching(n_ues=8, n_slots_trace=2)
    xs = [inputs.make_iq(3, sp, 3) for sp in specs]
    base, _ = _stream(specs, xs, 3, dict(persistent=True))
    tuned, _ = _stream(specs, xs, 3, dict(persistent=True, graphs=True), autotune=True)
    for a, b in zip(base, tuned):
        assert np.array_equal(a, b)
    for s in (1, 2, 4, 16):
        other = run_gpu(specs[:3], xs[:3], 3, spt=s)
        for a, b in zip(base[:3], other):
            assert np.array_equal(a, b)


def _run_per_slot(specs, xs, n_slots, per_run, cf32, ring_extra):
    """One engine as the batching benchmark builds it (CUDA graphs, persistent CTAs, autotuned),
    per_run slots of every UE per run, every UE's output pulled after each run."""
    eng = tc.Engine(graphs=True, persistent=True)
    chans = [tc.Chan(eng, sp, ring_slots=hist_slots(sp) + ring_extra, cf32=cf32) for sp in specs]
    assert eng.autotune(reps=2) >= 0
    outs = [[] for _ in specs]
    for s in range(0, n_slots, per_run):
        for ch, x in zip(chans, xs):
            ch.push(s, tc.slots_major(x, ch.n)[s:s + per_run])
        eng.run()
        for i, ch in enumerate(chans):
            outs[i].append(ch.pull(s, per_run))
    st = eng.stats()
    eng.close()
    return [tc.antenna_major(np.concatenate(o, 0)) for o in outs], st


def test_full_size_256_mixed_ues_against_oracle():
    """All 256 UEs of the batching workload (5/20/40/100 MHz 1:2:4:1, 4-48 taps, delays <= 512, AWGN
    20 dB) for 3 slots, one slot of every UE per run as the benchmark runs them (the graph replays from
    the second run on).  Every UE against the oracle: complex64 NRMSE and int16 within one LSB."""
    from tests.test_parity_gpu import assert_int16_close
    specs = inputs.workload_batching(n_ues=256, n_slots_trace=4)
    xs = [inputs.make_iq(3, sp, 3) for sp in specs]
    refs = [oracle.run_ue(oracle.OracleUE.from_spec(sp), x) for sp, x in zip(specs, xs)]
    ys, st = _run_per_slot(specs, xs, 3, 1, True, 4)
    assert st["graph_launches"] >= 2
    for y, (y_ref, _) in zip(ys, refs):
        assert nrmse(y, y_ref) <= 1e-5
    qs, _ = _run_per_slot(specs, xs, 3, 1, False, 4)
    for q, (y_ref, q_ref) in zip(qs, refs):
        assert_int16_close(q, y_ref, q_ref)


def test_eight_mixed_ues_over_200_slots_against_oracle():
    """8 UEs of the batching workload over 200 slots (looping 20-slot traces replayed ten times),
    20 slots per run: the trace cursors, delay lines and graph replays stay exact over a long run."""
    specs = inputs.workload_batching(n_ues=8, n_slots_trace=20)
    xs = [inputs.make_iq(3, sp, 200) for sp in specs]
    ys, _ = _run_per_slot(specs, xs, 200, 20, True, 21)
    for sp, x, y in zip(specs, xs, ys):
        y_ref, _ = oracle.run_ue(oracle.OracleUE.from_spec(sp), x)
        assert nrmse(y, y_ref) <= 1e-5


def _replay_last_outputs(specs, xs, steps, engine_kw, chan_kw=None):
    """The benchmark's replay (slot 0 pushed, then `steps` slot-synchronous steps that commit each
    UE's next slot in place and release the previous ones at launch) on the smallest ring the
    engine admits (two slots beyond the delay line); returns every UE's last output slot."""
    eng = tc.Engine(persistent=True, **engine_kw)
    try:
        chans = [tc.Chan(eng, sp, ring_slots=hist_slots(sp) + 2, **(chan_kw or {})) for sp in specs]
        for ch, x in zip(chans, xs):
            ch.push(0, tc.slots_major(x, ch.n)[:1])
        eng.run()
        tc.tt_engine_replay(eng.h, steps, 1)
        return [ch.pull(steps, 1) for ch in chans]         # the last step's slot (not yet released)
    finally:
        eng.close()


def test_replays_on_launch_lanes_equal_one_stream_on_a_minimal_ring():
    """Graph replays rotate over four launch lanes, so consecutive steps overlap on the GPU.  A
    replay releases each step's outputs at launch, so on the smallest ring every step rewrites the
    output position of the step one ring depth (3 to 4 slots here) earlier, which may still run
    on another lane: the writes must still land in launch order.  Against the same replay on one
    stream (direct launches), bit for bit."""
    specs = inputs.workload_batching(n_ues=12, n_slots_trace=2)
    xs = [inputs.make_iq(9, sp, 1) for sp in specs]
    one = _replay_last_outputs(specs, xs, 64, dict())
    lanes = _replay_last_outputs(specs, xs, 64, dict(graphs=True))
    for a, b in zip(one, lanes):
        assert np.array_equal(a, b)


def test_tensor_core_replays_on_launch_lanes_equal_one_stream():
    """The same for tensor-core channels (BF16, 4x4, dense taps), whose kernels of consecutive slots
    overlap on the lanes of a graph-replaying engine: bit for bit against one stream."""
    specs = [inputs.make_ue(17, u, 1024, 48, 95, 100.0, 2, n_tx=4 if u % 2 else 2, n_rx=4, pdp="per_tap",
                            delays=list(range(48))) for u in range(6)]
    xs = [inputs.make_iq(17, sp, 1) for sp in specs]
    kw = dict(precision=tc.TT_BF16_TC, cf32=True)
    one = _replay_last_outputs(specs, xs, 48, dict(), kw)
    lanes = _replay_last_outputs(specs, xs, 48, dict(graphs=True), kw)
    for a, b in zip(one, lanes):
        assert np.array_equal(a, b)


def _replay_steps(specs, xs, steps, k, engine_kw, make_chan):
    """The benchmark's replay with k slots per step (the first k pushed, then `steps` steps that
    commit k slots per UE in place and release the previous ones at launch) on a ring of
    k + hist + 1 slots; returns every UE's last k output slots."""
    eng = tc.Engine(persistent=True, **engine_kw)
    try:
        chans = [make_chan(eng, sp, k + hist_slots(sp) + 1) for sp in specs]
        for ch, x in zip(chans, xs):
            ch.push(0, tc.slots_major(x, ch.n)[:k])
        eng.run()
        tc.tt_engine_replay(eng.h, steps, k)
        return [ch.pull(steps * k, k) for ch in chans]
    finally:
        eng.close()


def _synthesised_chan(eng, sp, ring):
    ch = tc.Chan(eng, sp, ring_slots=ring, load=False)
    rng = np.random.default_rng([0x7717000B, sp.ue_id])
    amp, freq, phase = inputs.sos_params(rng, 300.0, inputs.pdp_span_decay(sp.delays, 20.0), sp.n_rx, sp.n_tx)
    tc.tt_chan_load_jakes(ch.h, sp.delays, amp, freq, phase, sp.fs)
    return ch


@pytest.mark.parametrize("kind", ["synthesised", "timed_1ms", "top_n"])
def test_replays_with_anchor_prepasses_on_launch_lanes_equal_one_stream(kind):
    """Synthesised, 1 ms-timed and top-n channels rewrite their anchor (or sparse-tap) ring before
    each run, on the engine stream.  With 4 slots per step on a ring of 4 + hist + 1 slots, each
    step's pre-pass rewrites ring positions whose earlier anchors the previous step reads, and that
    step may still run on another launch lane: the rewrite must wait for it.  Graph replays on four
    lanes against the same replay on one stream, bit for bit."""
    k, steps = 4, 24
    if kind == "timed_1ms":      # 20 MHz: one trace entry per 30720 samples (1 ms)
        specs = [inputs.make_ue(19, u, 1024, 12, 100, 300.0, 8, n_rx=1 + u % 2, loop=True,
                                step_samples=30720.0) for u in range(8)]
    else:
        specs = [inputs.make_ue(19, u, 1024, 16, 100, 300.0, 8, n_rx=1 + u % 2, loop=True) for u in range(8)]
    xs = [inputs.make_iq(19, sp, k) for sp in specs]
    if kind == "synthesised":
        make = _synthesised_chan
    elif kind == "top_n":
        def make(eng, sp, ring):
            return tc.Chan(eng, sp, ring_slots=ring, top_n=5)
    else:
        def make(eng, sp, ring):
            return tc.Chan(eng, sp, ring_slots=ring)
    one = _replay_steps(specs, xs, steps, k, dict(), make)
    lanes = _replay_steps(specs, xs, steps, k, dict(graphs=True), make)
    for a, b in zip(one, lanes):
        assert np.array_equal(a, b)
