"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bars: FP32 pre-pack output (TT_OUT_CF32) within NRMSE 1e-5 of the oracle's y;
int16 output within +-1 LSB of the oracle's q, with every mismatch sitting at a
rounding tie (|frac(y) - 0.5| < 0.01) or at saturation; bit-exact where every
product and sum is exact in FP32 (integer taps and inputs).
"""
import zlib

import numpy as np
import pytest

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.gpu_harness import run_gpu
from tests.helpers import nrmse

pytestmark = pytest.mark.gpu

NRMSE_MAX = 1e-5


class Spec:
    """Minimal UE description for hand-made cases (same fields as inputs.UESpec)."""

    def __init__(self, L, n_tx, n_rx, delays, taps, step=0.0, loop=False, noise_var=0.0, seed=7, ue_id=0,
                 max_delay=None):
        self.symbol_len = list(L)
        self.n_tx, self.n_rx = n_tx, n_rx
        self.delays = np.asarray(delays, dtype=np.int32)
        self.taps = np.asarray(taps, dtype=np.complex64)
        self.step_samples = float(step)
        self.loop = loop
        self.noise_var = float(noise_var)
        self.seed = seed
        self.ue_id = ue_id
        self.max_delay = int(self.delays.max()) if max_delay is None else max_delay

    @property
    def n(self):
        return int(sum(self.symbol_len))


def _taps(rng, T, n_rx, n_tx, K):
    z = rng.standard_normal((T, n_rx, n_tx, K)) + 1j * rng.standard_normal((T, n_rx, n_tx, K))
    return (z / np.sqrt(2 * K * n_tx)).astype(np.complex64)


def _case(name):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    if name == "siso_odd_lengths":
        L, nt, nr, d, ns, step, loop, nv = [7, 6, 6, 6], 1, 1, [0, 1, 5, 13], 5, 0, False, 0.0
    elif name == "delay_beyond_slot":
        L, nt, nr, d, ns, step, loop, nv = [10, 8, 8, 8], 1, 1, [0, 3, 40, 77], 6, 0, True, 0.0
    elif name == "mimo22_noise":
        L, nt, nr, d, ns, step, loop, nv = [16, 16, 16, 16], 2, 2, [0, 2, 9, 17, 30], 4, 0, False, 500.0
    elif name == "mimo_4tx_3rx_tracetime":
        L, nt, nr, d, ns, step, loop, nv = [24, 24], 4, 3, list(range(8)), 5, 11.5, False, 0.0
    elif name == "nr5mhz_loop_noise":
        L = inputs.nr_symbol_lengths(256)
        nt, nr, ns, step, loop, nv = 1, 1, 3, 0, True, inputs.noise_var_for_snr(20.0)
        d = inputs.gen_delays(rng, 20, 512)
    elif name == "nr20mhz_mimo_1ms_trace":
        L = inputs.nr_symbol_lengths(1024)
        nt, nr, ns, step, loop, nv = 2, 2, 3, 30720.0, False, inputs.noise_var_for_snr(10.0)
        d = inputs.gen_delays(rng, 12, 300)
    else:
        raise KeyError(name)
    n = sum(L)
    if step:
        T = int(np.ceil(ns * n / step)) + 3
    else:
        T = (len(L) * ns + 1) if not loop else len(L) + 3
    taps = _taps(rng, T, nr, nt, len(d))
    spec = Spec(L, nt, nr, d, taps, step, loop, nv, seed=0xABCDEF12345, ue_id=3)
    x = np.clip(np.rint(rng.standard_normal((nt, ns * n, 2)) * 1024), -32768, 32767).astype(np.int16)
    return spec, x, ns


CASES = ["siso_odd_lengths", "delay_beyond_slot", "mimo22_noise", "mimo_4tx_3rx_tracetime",
         "nr5mhz_loop_noise", "nr20mhz_mimo_1ms_trace"]
VARIANTS = [dict(form="batched"), dict(form="batched", persistent=True), dict(form="batched", spt=1),
            dict(form="batched", spt=2), dict(form="batched", spt=16), dict(form="plain"),
            # 256 threads per CTA: work items twice as long
            dict(form="batched", tpb=256), dict(form="batched", spt=1, tpb=256),
            dict(form="batched", persistent=True, spt=16, tpb=256)]


def _oracle(spec, x, first_slot=0):
    return oracle.run_ue(oracle.OracleUE.from_spec(spec), x, s_first=first_slot)


def assert_int16_close(q, y_ref, q_ref):
    diff = np.abs(q.astype(np.int32) - q_ref.astype(np.int32))
    assert diff.max() <= 1
    bad = np.nonzero(diff)
    if bad[0].size:
        comp = np.stack([y_ref.real, y_ref.imag], axis=-1)[bad]
        frac = np.abs(np.abs(comp - np.floor(comp)) - 0.5)
        assert np.all((frac < 0.01) | (np.abs(comp) > 32766.5)), "int16 mismatch away from a rounding tie"


@pytest.mark.parametrize("variant", range(len(VARIANTS)))
@pytest.mark.parametrize("case", CASES)
def test_small_cases_match_oracle(case, variant):
    spec, x, ns = _case(case)
    first = 5
    y_ref, q_ref = _oracle(spec, x, first)
    kw = VARIANTS[variant]
    y = run_gpu([spec], [x], ns, first_slot=first, cf32=True, **kw)[0]
    assert nrmse(y, y_ref) <= NRMSE_MAX
    q = run_gpu([spec], [x], ns, first_slot=first, cf32=False, **kw)[0]
    assert_int16_close(q, y_ref, q_ref)


def test_integer_taps_and_impulses_are_bit_exact():
    """Small integer taps, integer impulses crossing slot boundaries: exact in FP32, so bit-exact."""
    rng = np.random.default_rng(21)
    L = inputs.nr_symbol_lengths(256)
    n = sum(L)
    d = np.array([0, 3, 7, 12, 20, 40, 300, 511], dtype=np.int32)
    h = (rng.integers(-3, 4, size=(1, 2, 2, len(d))) + 1j * rng.integers(-3, 4, size=(1, 2, 2, len(d))))
    taps = np.repeat(h, 14 * 4 + 1, axis=0).astype(np.complex64)
    spec = Spec(L, 2, 2, d, taps)
    x = np.zeros((2, 3 * n, 2), dtype=np.int16)
    for m0 in (0, 1, n - 1, n, n + 7, 2 * n - 1, 2 * n - 300):
        x[0, m0] = (rng.integers(-900, 900), rng.integers(-900, 900))
        x[1, m0] = (rng.integers(-900, 900), rng.integers(-900, 900))
    x[:, 2 * n + 10:2 * n + 500] = rng.integers(-1000, 1000, size=(2, 490, 2))
    y_ref, q_ref = _oracle(spec, x, 0)
    for kw in VARIANTS:
        q = run_gpu([spec], [x], 3, cf32=False, **kw)[0]
        assert np.array_equal(q, q_ref), kw
        y = run_gpu([spec], [x], 3, cf32=True, **kw)[0]
        assert np.array_equal(y.astype(np.complex128), y_ref), kw


def test_stream_mode_ring_wrap_equals_bulk():
    spec, x, _ = _case("delay_beyond_slot")
    rng = np.random.default_rng(5)
    ns = 12
    spec.taps = _taps(rng, 4 * ns + 1, 1, 1, len(spec.delays))
    spec.loop = False
    x = rng.integers(-2000, 2000, size=(1, ns * spec.n, 2)).astype(np.int16)
    y_ref, q_ref = _oracle(spec, x, 0)
    bulk = run_gpu([spec], [x], ns, cf32=False)[0]
    stream = run_gpu([spec], [x], ns, cf32=False, stream_mode=True)[0]
    assert np.array_equal(bulk, stream)
    assert_int16_close(stream, y_ref, q_ref)


def test_each_result_is_the_same_alone_and_in_the_mix():
    specs = inputs.workload_batching(n_ues=12, n_slots_trace=2)
    xs = [inputs.make_iq(3, sp, 2) for sp in specs]
    mix = run_gpu(specs, xs, 2, cf32=True)
    for i in (0, 3, 7, 11):
        alone = run_gpu([specs[i]], [xs[i]], 2, cf32=True)[0]
        assert np.array_equal(alone, mix[i])
    mix_p = run_gpu(specs, xs, 2, cf32=True, persistent=True)
    for i in range(len(specs)):
        assert np.array_equal(mix_p[i], mix[i])


def test_checkpoint_resume_is_bit_identical():
    spec = inputs.make_ue(2, 1, 1024, 10, 200, 100.0, 8, snr_db=20.0)
    x = inputs.make_iq(2, spec, 8)
    straight = run_gpu([spec], [x], 8, cf32=False)[0]
    eng = tc.Engine()
    ch = tc.Chan(eng, spec, ring_slots=6)
    xs = tc.slots_major(x, spec.n)
    ch.push(0, xs[:4])
    eng.run()
    a = ch.pull(0, 4)
    eng.sync()
    blob = tc.tt_chan_get_state(ch.h)
    eng.close()
    eng2 = tc.Engine()
    ch2 = tc.Chan(eng2, spec, ring_slots=6)
    tc.tt_chan_set_state(ch2.h, blob)
    ch2.push(4, xs[4:])
    eng2.run()
    b = ch2.pull(4, 4)
    eng2.close()
    resumed = tc.antenna_major(np.concatenate([a, b], axis=0))
    assert np.array_equal(resumed, straight)


def test_workload_plain_1ue_all_slots():
    """1 UE SISO, 20 MHz, 10 slots, taps {0,3,7,12,20,40}, 3 dB/tap, 10 Hz Jakes, no AWGN."""
    spec = inputs.workload_plain_1ue(10)[0]
    x = inputs.make_iq(1, spec, 10)
    y_ref, q_ref = _oracle(spec, x)
    for kw in (dict(form="batched"), dict(form="plain")):
        y = run_gpu([spec], [x], 10, cf32=True, **kw)[0]
        assert nrmse(y, y_ref) <= NRMSE_MAX
        q = run_gpu([spec], [x], 10, cf32=False, **kw)[0]
        assert_int16_close(q, y_ref, q_ref)


def test_workload_plain_16ue_full_size_sampled_slots():
    """16 UEs x 1000 slots at 40 MHz, 24 taps <= 256, 100 Hz, SNR 20 dB, run as the benchmark runs it
    (every slot of every UE in one batched launch); checked on slots 0-49 and 990-999 of every UE.
    The last configuration is the benchmark's own: persistent CTAs, 16 samples per thread, int16 out."""
    specs = inputs.workload_plain_16ue(1000)
    n = specs[0].n
    xs = [inputs.make_iq(2, sp, 1000) for sp in specs]
    refs = []
    for sp, x in zip(specs, xs):
        y0, q0 = _oracle(sp, x[:, : 50 * n])
        y1, q1 = _oracle(sp, x[:, 989 * n:], first_slot=989)
        refs.append((y0, q0, y1[:, n:], q1[:, n:]))
    configs = [(dict(form="batched"), True), (dict(form="batched", persistent=True), True),
               (dict(form="batched", persistent=True, samples_per_thread=16), True),
               (dict(form="batched", persistent=True, samples_per_thread=16), False)]
    for kw, cf32 in configs:
        eng = tc.Engine(**kw)
        chans = [tc.Chan(eng, sp, ring_slots=1002, cf32=cf32) for sp in specs]
        for ch, x in zip(chans, xs):
            ch.push(0, x)
        eng.run()
        for ch, (y0, q0, y1, q1) in zip(chans, refs):
            out = tc.antenna_major(ch.pull(0, 1000))
            if cf32:
                assert nrmse(out[:, : 50 * n], y0) <= NRMSE_MAX
                assert nrmse(out[:, 990 * n:], y1) <= NRMSE_MAX
            else:
                assert_int16_close(out[:, : 50 * n], y0, q0)
                assert_int16_close(out[:, 990 * n:], y1, q1)
        eng.close()


def test_largest_channels():
    """4x4 MIMO at 100 MHz: 128 taps up to a 512-sample delay run (the kernel picks the geometry that
    fits shared memory); 128 taps with delays up to 1024 do not fit and are refused cleanly."""
    rng = np.random.default_rng(9)
    L = inputs.nr_symbol_lengths(4096)
    d = np.concatenate([[0], np.sort(rng.choice(np.arange(1, 513), 127, replace=False))]).astype(np.int32)
    spec = Spec(L, 4, 4, d, _taps(rng, 30, 4, 4, 128), loop=True, noise_var=100.0)
    x = rng.integers(-3000, 3000, size=(4, 2 * sum(L), 2)).astype(np.int16)
    y_ref, _ = _oracle(spec, x)
    y = run_gpu([spec], [x], 2, cf32=True)[0]
    assert nrmse(y, y_ref) <= NRMSE_MAX
    d2 = np.concatenate([[0], np.sort(rng.choice(np.arange(1, 1025), 127, replace=False))]).astype(np.int32)
    big = Spec(L, 4, 4, d2, _taps(rng, 30, 4, 4, 128), loop=True)
    eng = tc.Engine()
    with pytest.raises(tc.TTError) as ei:
        tc.Chan(eng, big, ring_slots=4)
    assert ei.value.status == tc.TT_ERR_INVALID
    eng.close()


def test_dense_96tap_4x4_channel():
    """The dense 4x4 x 96-tap (delays 0..95) channel of the precision workload on the FP32 path."""
    spec = inputs.workload_precision(n_ues=1, n_slots_trace=2)[0]
    x = inputs.make_iq(4, spec, 2)
    y_ref, q_ref = _oracle(spec, x)
    y = run_gpu([spec], [x], 2, cf32=True)[0]
    assert nrmse(y, y_ref) <= NRMSE_MAX
    q = run_gpu([spec], [x], 2, cf32=False)[0]
    assert_int16_close(q, y_ref, q_ref)


def test_errors_and_admission():
    eng = tc.Engine(hbm_budget_bytes=4 << 20)
    spec = inputs.make_ue(2, 0, 1024, 6, 40, 10.0, 2)
    ch = tc.Chan(eng, spec, ring_slots=8)     # 8 * 15360 * 8 B = 983 KB
    with pytest.raises(tc.TTError) as ei:
        tc.Chan(eng, spec, ring_slots=64)     # 7.9 MB: over the budget
    assert ei.value.status == tc.TT_ERR_NO_MEMORY
    with pytest.raises(tc.TTError) as ei:
        tc.tt_chan_load_trace(ch.h, spec.taps, np.array([0, 3, 2, 5, 6, 7]))
    assert ei.value.status == tc.TT_ERR_TRACE
    bad = spec.taps.copy()
    bad[0, 0, 0, 0] = np.nan
    with pytest.raises(tc.TTError) as ei:
        tc.tt_chan_load_trace(ch.h, bad, spec.delays)
    assert ei.value.status == tc.TT_ERR_TRACE
    x = tc.slots_major(inputs.make_iq(2, spec, 8), spec.n)
    ch.push(3, x[:2])
    with pytest.raises(tc.TTError) as ei:
        ch.push(7, x[2:3])                    # out of order
    assert ei.value.status == tc.TT_ERR_STATE
    ch.push(5, x[2:7])                        # 7 slots pushed, ring of 8 with 1 history slot: full
    with pytest.raises(tc.TTError) as ei:
        ch.push(10, x[7:8])
    assert ei.value.status == tc.TT_ERR_AGAIN
    with pytest.raises(tc.TTError) as ei:
        ch.pull(3, 1, timeout_us=0)           # not launched
    assert ei.value.status == tc.TT_ERR_AGAIN
    eng.run()
    ch.pull(3, 7)
    ch.push(10, x[7:8])                       # room again
    tc.tt_chan_push_slots(ch.h, 11, 0, None)  # empty push is a no-op
    eng.run()
    eng.run()                                 # nothing pending: no-op
    ch.pull(10, 1)
    st = eng.stats()
    assert st["n_chans"] == 1 and st["hbm_in_use"] > 0 and st["slots_processed"] == 8
    cell = tc.Cell(eng, 0, spec.n, n_rx=spec.n_rx, ring_slots=8)
    eng.close()                               # frees the channel and the cell with the engine
    ch.destroy()                              # handles were cleared: no call on freed memory
    cell.destroy()
    with pytest.raises(tc.TTError) as ei:
        ch.push(11, x[:1])
    assert ei.value.status == tc.TT_ERR_INVALID
    with pytest.raises(tc.TTError) as ei:
        cell.pull(0, 1, timeout_us=0)
    assert ei.value.status == tc.TT_ERR_INVALID


def test_device_buffers_and_zero_copy_paths():
    import torch
    spec = inputs.make_ue(2, 2, 2048, 8, 100, 50.0, 3, n_tx=2, n_rx=2, snr_db=15.0)
    x = inputs.make_iq(2, spec, 3)
    ref = run_gpu([spec], [x], 3, cf32=False)[0]
    xs = tc.slots_major(x, spec.n)
    eng = tc.Engine()
    ch = tc.Chan(eng, spec, ring_slots=6)
    dev = torch.from_numpy(xs).cuda()
    s = torch.cuda.current_stream()
    tc.tt_chan_push_slots_dev(ch.h, 0, 2, dev[:2], s)
    p = tc.tt_chan_slot_input(ch.h, 2)        # zero-copy: write slot 2 straight into the ring
    dst = torch.empty(xs[2].size, dtype=torch.int16, device="cuda")
    dst.copy_(dev[2].reshape(-1))
    torch.cuda.synchronize()
    import ctypes
    cudart = ctypes.CDLL("libcudart.so.13")
    assert cudart.cudaMemcpy(ctypes.c_void_p(p), ctypes.c_void_p(dst.data_ptr()),
                             ctypes.c_size_t(xs[2].nbytes), 3) == 0
    tc.tt_chan_commit_slots(ch.h, 2, 1)
    eng.run()
    out = torch.empty((2,) + xs.shape[1:2] + (spec.n, 2), dtype=torch.int16, device="cuda")
    tc.tt_chan_pull_slots_dev(ch.h, 0, 2, out, s)
    eng.sync()
    op = tc.tt_chan_slot_output(ch.h, 2)
    last = torch.empty((1, 2, spec.n, 2), dtype=torch.int16, device="cuda")
    assert cudart.cudaMemcpy(ctypes.c_void_p(last.data_ptr()), ctypes.c_void_p(op),
                             ctypes.c_size_t(last.numel() * 2), 3) == 0
    tc.tt_chan_release_slots(ch.h, 2, 1)
    got = torch.cat([out, last], 0).cpu().numpy()
    assert np.array_equal(tc.antenna_major(got), ref)
    eng.close()

    # the single-slot device calls and the slot-synchronous run: slot by slot, device buffers only
    eng = tc.Engine()
    ch = tc.Chan(eng, spec, ring_slots=4)
    outs = torch.empty((3,) + xs.shape[1:2] + (spec.n, 2), dtype=torch.int16, device="cuda")
    for k in range(3):
        tc.tt_chan_push_slot_dev(ch.h, k, dev[k], s)
        tc.tt_engine_run_slot(eng.h)
        assert tc.tt_chan_pull_slot_dev(ch.h, outs[k], s) == k
    with pytest.raises(tc.TTError) as ei:
        tc.tt_chan_pull_slot_dev(ch.h, outs[0], s)        # nothing launched past slot 2
    assert ei.value.status == tc.TT_ERR_AGAIN
    torch.cuda.synchronize()
    assert np.array_equal(tc.antenna_major(outs.cpu().numpy()), ref)
    eng.close()


def test_producer_and_consumer_threads_on_one_channel_equal_bulk():
    """One thread pushes and launches slot after slot while another pulls them, on the same
    channels, through a ring only a few slots deep: the output equals the bulk run bit for bit,
    and the ring-full refusal (TT_ERR_AGAIN) is the producer's only back-pressure."""
    import threading
    import time
    specs = inputs.workload_plain_16ue(n_slots=12, n_ues=3)
    xs = [inputs.make_iq(2, sp, 12) for sp in specs]
    bulk = run_gpu(specs, xs, 12)
    eng = tc.Engine(persistent=True)
    try:
        from tests.gpu_harness import hist_slots
        chans = [tc.Chan(eng, sp, ring_slots=hist_slots(sp) + 3) for sp in specs]
        outs = [[None] * 12 for _ in specs]
        launched = []
        lock = threading.Condition()
        err = []

        def producer():
            try:
                for s in range(12):
                    for ch, x in zip(chans, xs):
                        while True:
                            try:
                                ch.push(s, tc.slots_major(x, ch.n)[s:s + 1])
                                break
                            except tc.TTError as ex:
                                if ex.status != tc.TT_ERR_AGAIN:
                                    raise
                                time.sleep(1e-4)
                    eng.run()
                    with lock:
                        launched.append(s)
                        lock.notify()
            except Exception as ex:
                err.append(ex)
                with lock:
                    launched.append(None)
                    lock.notify()

        th = threading.Thread(target=producer)
        th.start()
        for s in range(12):
            with lock:
                lock.wait_for(lambda: len(launched) > s)
                if launched[s] is None:
                    break
            for i, ch in enumerate(chans):
                outs[i][s] = ch.pull(s, 1)
        th.join()
        assert not err, err
        for i in range(len(specs)):
            got = tc.antenna_major(np.concatenate(outs[i], axis=0))
            assert np.array_equal(got, bulk[i])
    finally:
        eng.close()


def test_many_channel_push_and_pull_equal_per_channel_calls():
    """tt_engine_push_slots / tt_engine_pull_slots move every channel's slots in one call and give
    the same bits as per-channel calls; a repeated channel or an out-of-order slot is refused
    before anything is copied."""
    specs = inputs.workload_plain_16ue(n_slots=6, n_ues=3)
    xs = [tc.slots_major(inputs.make_iq(2, sp, 6), sp.n) for sp in specs]
    bulk = run_gpu(specs, [inputs.make_iq(2, sp, 6) for sp in specs], 6)
    eng = tc.Engine(persistent=True)
    try:
        chans = [tc.Chan(eng, sp, ring_slots=10) for sp in specs]
        hs = [ch.h for ch in chans]
        with pytest.raises(tc.TTError) as ex:
            tc.tt_engine_push_slots(eng.h, [hs[0], hs[0]], [0, 0], [3, 3], [xs[0], xs[0]])
        assert ex.value.status == tc.TT_ERR_INVALID
        outs = [np.zeros((6, 1, sp.n, 2), dtype=np.int16) for sp in specs]
        for s0 in (0, 3):
            bufs = [np.ascontiguousarray(x[s0:s0 + 3]) for x in xs]
            tc.tt_engine_push_slots(eng.h, hs, [s0] * 3, [3] * 3, bufs)
            eng.run()
        with pytest.raises(tc.TTError) as ex:
            tc.tt_engine_pull_slots(eng.h, hs, [3] * 3, [3] * 3, [o[3:] for o in outs])
        assert ex.value.status == tc.TT_ERR_STATE
        for s0 in (0, 3):
            part = [np.zeros((3, 1, sp.n, 2), dtype=np.int16) for sp in specs]
            tc.tt_engine_pull_slots(eng.h, hs, [s0] * 3, [3] * 3, part)
            for o, p in zip(outs, part):
                o[s0:s0 + 3] = p
        for i in range(3):
            assert np.array_equal(tc.antenna_major(outs[i]), bulk[i])
    finally:
        eng.close()


def test_saturation_is_bit_exact():
    """Full-scale int16 input through integer taps with gain above one: most outputs clamp to
    -32768 or 32767.  Every product and sum is exact in FP32, so the packed output is bit-exact."""
    rng = np.random.default_rng(31)
    L = inputs.nr_symbol_lengths(256)
    n = sum(L)
    d = np.array([0, 1, 5], dtype=np.int32)
    h = np.array([3 + 2j, -2 + 1j, 1 - 3j]).reshape(1, 1, 1, 3)
    spec = Spec(L, 1, 1, d, np.repeat(h, 14 * 2 + 1, axis=0))
    x = rng.integers(-32768, 32768, size=(1, 2 * n, 2)).astype(np.int16)
    _, q_ref = _oracle(spec, x)
    assert np.mean((q_ref == 32767) | (q_ref == -32768)) > 0.5
    for kw in VARIANTS:
        q = run_gpu([spec], [x], 2, cf32=False, **kw)[0]
        assert np.array_equal(q, q_ref), kw


def test_single_tap_and_noise_only_cases():
    """K = 1 at d = 0 (y = h(m) x(m), the paper's per-symbol scaling case), and zero input with AWGN
    on (the output is the noise alone) for a 2x2 channel."""
    rng = np.random.default_rng(32)
    L = inputs.nr_symbol_lengths(1024)
    n = sum(L)
    a = np.arange(14 * 2 + 1)
    g = 10.0 ** (-6.0 * (1 - np.cos(2 * np.pi * a / 9.0)) / 20.0)     # periodic SNR-degradation gain
    spec = Spec(L, 1, 1, [0], (g * np.exp(0.3j * a)).reshape(-1, 1, 1, 1))
    x = rng.integers(-3000, 3000, size=(1, 2 * n, 2)).astype(np.int16)
    y_ref, q_ref = _oracle(spec, x)
    y = run_gpu([spec], [x], 2, cf32=True)[0]
    assert nrmse(y, y_ref) <= NRMSE_MAX
    assert_int16_close(run_gpu([spec], [x], 2)[0], y_ref, q_ref)
    # the output power follows the trace's gain: |y|^2 / |x|^2 = |h(m)|^2, between 1 and -12 dB
    xc = x[0, :, 0].astype(np.float64) + 1j * x[0, :, 1]
    nz = np.abs(xc) > 0
    gain_db = 10 * np.log10(np.abs(y[0][nz]) ** 2 / np.abs(xc[nz]) ** 2)
    assert gain_db.max() < 1e-3 and gain_db.min() > -12.0 - 1e-3 and gain_db.min() < -10.0
    noisy = Spec(L, 2, 2, [0, 4, 9], _taps(rng, 14 * 2 + 1, 2, 2, 3), noise_var=2.0 ** 21 / 100, ue_id=9)
    z = np.zeros((2, 2 * n, 2), dtype=np.int16)
    y_ref, q_ref = _oracle(noisy, z)
    assert np.std(y_ref) > 50
    assert nrmse(run_gpu([noisy], [z], 2, cf32=True)[0], y_ref) <= NRMSE_MAX
    assert_int16_close(run_gpu([noisy], [z], 2)[0], y_ref, q_ref)


def test_maximum_delay_and_maximum_slot_size():
    """The largest delay class (d = 1024) at 5 MHz, where the delay line spans a quarter slot, and the
    largest slot (2^24 samples in 32 symbols of 2^19) with a short channel."""
    rng = np.random.default_rng(33)
    L = inputs.nr_symbol_lengths(256)
    spec = Spec(L, 1, 1, [0, 511, 1000, 1024], _taps(rng, 14 * 3 + 1, 1, 1, 4), noise_var=100.0)
    x = rng.integers(-3000, 3000, size=(1, 3 * spec.n, 2)).astype(np.int16)
    y_ref, q_ref = _oracle(spec, x)
    for kw in (dict(form="batched", persistent=True), dict(form="plain")):
        assert nrmse(run_gpu([spec], [x], 3, cf32=True, **kw)[0], y_ref) <= NRMSE_MAX
        assert_int16_close(run_gpu([spec], [x], 3, **kw)[0], y_ref, q_ref)
    big = Spec([1 << 19] * 32, 1, 1, [0, 7], _taps(rng, 32 * 2 + 1, 1, 1, 2))
    assert big.n == 1 << 24
    xb = rng.integers(-3000, 3000, size=(1, 2 * big.n, 2)).astype(np.int16)
    y_ref, q_ref = _oracle(big, xb)
    yb = run_gpu([big], [xb], 2, cf32=True, persistent=True)[0]
    assert nrmse(yb, y_ref) <= NRMSE_MAX
    del yb
    assert_int16_close(run_gpu([big], [xb], 2, persistent=True)[0], y_ref, q_ref)
