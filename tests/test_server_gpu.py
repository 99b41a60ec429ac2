"""Serving with callers' own pushes (continuous batching of slot requests as they arrive).

An engine-owned batching thread (tt_server_start) launches whatever producer threads push, host and
device buffers alike, at Poisson times.  Bars:
- every UE's output equals the same UE run alone, bit for bit (per-UE isolation, Sec. III-C);
- every UE's output also meets the oracle's bars;
- a full ring queues the push instead of refusing it;
- the report's latencies come from device completion stamps;
- the admission waiting list admits channels in arrival order as destroyed channels free the budget.
"""
import threading
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.gpu_harness import hist_slots, run_gpu
from tests.test_parity_gpu import assert_int16_close

pytestmark = pytest.mark.gpu

N_SLOTS = 10


def _specs():
    out = []
    for u in range(6):
        n_fft = (1024, 256, 512)[u % 3]
        ant = 2 if u % 2 else 1
        out.append(inputs.make_ue(7, u, n_fft, 4 + 6 * u, 60 + 40 * u, 100.0, N_SLOTS + 2, n_tx=ant, n_rx=ant,
                                  snr_db=20.0))
    return out


@pytest.mark.parametrize("inflight", [2, 0])  # 0: the default, 8 batches on 8 launch lanes
def test_pushes_from_producer_threads_are_batched_and_match_alone_and_oracle(inflight):
    specs = _specs()
    xs = [inputs.make_iq(7, sp, N_SLOTS) for sp in specs]
    slots = [tc.slots_major(x, sp.n) for sp, x in zip(specs, xs)]
    eng = tc.Engine(form="batched", persistent=True)
    outs = [[None] * N_SLOTS for _ in specs]
    errors = []
    try:
        # rings two slots deeper than the delay line: producers outrun the consumer and must queue
        chans = [tc.Chan(eng, sp, ring_slots=hist_slots(sp) + 2) for sp in specs]
        dev = [torch.from_numpy(s).cuda() for s in slots]           # device copies for device pushes
        torch.cuda.synchronize()
        tc.tt_server_start(eng.h, max_inflight_batches=inflight, queue_timeout_us=10_000_000)

        def producer(ues, seed):
            rng = np.random.default_rng(seed)
            try:
                for s in range(N_SLOTS):
                    for u in ues:
                        time.sleep(rng.exponential(0.0005))
                        if u % 2 == 0:
                            tc.tt_chan_push_slot(chans[u].h, s, np.ascontiguousarray(slots[u][s]))
                        else:
                            tc.tt_chan_push_slot_dev(chans[u].h, s, dev[u][s], 0)
            except Exception as ex:  # surfaced after the join
                errors.append(ex)

        def consumer():
            try:
                left = {u: 0 for u in range(len(specs))}
                while left:
                    for u in list(left):
                        ch = chans[u]
                        try:
                            if u % 3 == 1:      # device pull: a copy ordered after the producing batch
                                d = torch.empty((1, ch.spec.n_rx, ch.n, 2), dtype=torch.int16, device="cuda")
                                st = torch.cuda.current_stream()
                                tc.tt_chan_pull_slots_dev(ch.h, left[u], 1, d, st)
                                st.synchronize()
                                buf = d.cpu().numpy()
                            else:
                                buf = np.empty((1, ch.spec.n_rx, ch.n, 2), dtype=np.int16)
                                tc.tt_chan_pull_slots(ch.h, left[u], 1, buf, -1)
                        except tc.TTError as ex:
                            if ex.status != tc.TT_ERR_AGAIN:
                                raise
                            continue
                        outs[u][left[u]] = buf[0]
                        left[u] += 1
                        if left[u] == N_SLOTS:
                            del left[u]
                    time.sleep(0.002)                                 # a slow consumer: rings fill
            except Exception as ex:
                errors.append(ex)

        threads = [threading.Thread(target=producer, args=([u for u in range(6) if u % 3 == p], 10 + p))
                   for p in range(3)]
        threads.append(threading.Thread(target=consumer))
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout=120)
        assert not errors, errors
        assert not any(t.is_alive() for t in threads)
        rep = tc.tt_server_stop(eng.h)
    finally:
        eng.close()
    assert rep["requests"] == rep["completed"] == 6 * N_SLOTS
    assert rep["refused"] == 0 and rep["queued"] > 0 and rep["batches"] >= 1
    assert 0 < rep["p50_us"] <= rep["p99_us"] <= rep["max_us"] and rep["stamp_error_us"] < 1000
    for u, (sp, x) in enumerate(zip(specs, xs)):
        served = tc.antenna_major(np.stack(outs[u]))
        alone = run_gpu([sp], [x], N_SLOTS)[0]
        assert np.array_equal(served, alone), u
        y_ref, q_ref = oracle.run_ue(oracle.OracleUE.from_spec(sp), x)
        assert_int16_close(served, y_ref, q_ref)


def test_a_push_whose_queue_wait_runs_out_is_refused():
    sp = _specs()[0]
    x = tc.slots_major(inputs.make_iq(7, sp, 6), sp.n)
    eng = tc.Engine()
    try:
        ch = tc.Chan(eng, sp, ring_slots=hist_slots(sp) + 2)
        tc.tt_server_start(eng.h, queue_timeout_us=20_000)
        tc.tt_chan_push_slot(ch.h, 0, np.ascontiguousarray(x[0]))
        tc.tt_chan_push_slot(ch.h, 1, np.ascontiguousarray(x[1]))
        t0 = time.perf_counter()
        with pytest.raises(tc.TTError) as ei:             # nothing pulls: the ring stays full
            tc.tt_chan_push_slot(ch.h, 2, np.ascontiguousarray(x[2]))
        assert ei.value.status == tc.TT_ERR_AGAIN and time.perf_counter() - t0 >= 0.015
        with pytest.raises(tc.TTError) as ei:             # the server launches the batches
            eng.run()
        assert ei.value.status == tc.TT_ERR_STATE
        rep = tc.tt_server_stop(eng.h)
    finally:
        eng.close()
    assert rep["requests"] == 2 and rep["queued"] == 1 and rep["refused"] == 1 and rep["completed"] == 2


def test_admission_waits_in_arrival_order_for_destroyed_channels():
    sp = _specs()[0]
    probe = tc.Engine()
    before = probe.stats()["hbm_in_use"]
    c0 = tc.Chan(probe, sp, ring_slots=4)
    one = probe.stats()["hbm_in_use"] - before                 # bytes of one such channel
    probe.close()
    eng = tc.Engine(hbm_budget_bytes=int(one * 1.5))
    order, errors = [], []
    try:
        a = tc.Chan(eng, sp, ring_slots=4)
        with pytest.raises(tc.TTError) as ei:                  # plain admission refuses
            tc.Chan(eng, sp, ring_slots=4)
        assert ei.value.status == tc.TT_ERR_NO_MEMORY
        with pytest.raises(tc.TTError) as ei:                  # a short wait runs out
            tc.Chan(eng, sp, ring_slots=4, wait_us=20_000)
        assert ei.value.status == tc.TT_ERR_NO_MEMORY
        got = {}

        def waiter(name):
            try:
                got[name] = tc.Chan(eng, sp, ring_slots=4, wait_us=30_000_000)
                order.append(name)
            except Exception as ex:
                errors.append(ex)

        tb = threading.Thread(target=waiter, args=("B",))
        tb.start()
        time.sleep(0.2)
        tcw = threading.Thread(target=waiter, args=("C",))
        tcw.start()
        time.sleep(0.2)
        assert order == []                                     # both wait
        a.destroy()
        tb.join(timeout=20)
        assert order == ["B"] and tcw.is_alive()                # B first, C still waits
        got["B"].destroy()
        tcw.join(timeout=20)
        assert order == ["B", "C"] and not errors
    finally:
        eng.close()
