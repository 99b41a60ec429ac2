"""The autotuner over samples per thread and threads per CTA, and its on-disk cache (TT_TUNE_CACHE).

Each output sample is accumulated in the same order whatever the kernel geometry, so every choice
must give the same bits.  Bars:
- tuning writes one line per channel class for this device model, keeps the lines of other device
  models and drops malformed ones;
- an engine created later reads the file: its channels start at the stored geometry, untuned, and
  their output equals the tuned engine's bit for bit;
- a stored 256-thread choice is taken, and its output equals the default 128-thread output bit for
  bit and meets the oracle's bars;
- a forced thread count (threads_per_block) wins over the cache and bounds the tuner;
- a cache path that cannot be written gives TT_ERR_IO, with the engine still correct.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.gpu_harness import hist_slots
from tests.test_parity_gpu import assert_int16_close

pytestmark = pytest.mark.gpu

N_SLOTS = 3
OTHER = "Some Other GPU\t100\tL=8;tx=1;rx=1;K=1;dc=0;awgn=0;cf32=0;top=0\t8\t256"


def _specs():
    out = []
    for u in range(6):
        n_fft = (1024, 512)[u % 2]
        ant = 2 if u % 3 == 2 else 1
        out.append(inputs.make_ue(11, u, n_fft, 8 + 4 * (u % 3), 100 + 50 * (u % 3), 100.0, N_SLOTS + 2,
                                  n_tx=ant, n_rx=ant, snr_db=20.0))
    return out


def _dclass(d):
    return 0 if d <= 128 else (1 if d <= 256 else (2 if d <= 512 else 3))


def _bucket(k):
    b = 8
    while b < k:
        b *= 2
    return b


def _classes(specs):
    return {(tuple(sp.symbol_len), sp.n_tx, sp.n_rx, _bucket(len(sp.delays)), _dclass(int(sp.delays.max())),
             sp.noise_var > 0) for sp in specs}


def _run(specs, xs, autotune=False, engine_kw=None):
    eng = tc.Engine(persistent=True, **(engine_kw or {}))
    try:
        chans = [tc.Chan(eng, sp, ring_slots=hist_slots(sp) + N_SLOTS + 2) for sp in specs]
        geo0 = [ch.geometry() for ch in chans]
        if autotune:
            eng.autotune(reps=2)
        geo = [ch.geometry() for ch in chans]
        for ch, x in zip(chans, xs):
            ch.push(0, tc.slots_major(x, ch.n))
        eng.run()
        outs = [tc.antenna_major(ch.pull(0, N_SLOTS)) for ch in chans]
        return outs, geo0, geo
    finally:
        eng.close()


def _ours(path):
    dev = torch.cuda.get_device_name(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    lines = path.read_text().splitlines()
    return [line.split("\t") for line in lines if line.startswith(f"{dev}\t{sms}\t")], lines


def test_tuned_choices_are_stored_and_reloaded(tmp_path, monkeypatch):
    specs = _specs()
    xs = [inputs.make_iq(11, sp, N_SLOTS) for sp in specs]
    path = tmp_path / "tune.tsv"
    path.write_text(OTHER + "\nnot a cache line\n")
    monkeypatch.setenv("TT_TUNE_CACHE", str(path))
    tuned, _, geo_tuned = _run(specs, xs, autotune=True)
    ours, lines = _ours(path)
    assert OTHER in lines and "not a cache line" not in lines
    assert len(ours) == len(_classes(specs)) == len(lines) - 1
    for f in ours:
        assert int(f[3]) in (1, 2, 4, 8, 16) and int(f[4]) in (128, 256)
    for g in geo_tuned:
        assert g["samples_per_item"] == g["samples_per_thread"] * g["threads_per_cta"]
    # a later engine starts every channel at the stored geometry, without tuning
    again, geo0, _ = _run(specs, xs)
    assert [(g["samples_per_thread"], g["threads_per_cta"]) for g in geo0] == \
           [(g["samples_per_thread"], g["threads_per_cta"]) for g in geo_tuned]
    for a, b in zip(tuned, again):
        assert np.array_equal(a, b)
    # and with no cache, the default geometry gives the same bits
    monkeypatch.delenv("TT_TUNE_CACHE")
    plain, geo_plain, _ = _run(specs, xs)
    assert all(g["threads_per_cta"] == 128 for g in geo_plain)
    for a, b in zip(tuned, plain):
        assert np.array_equal(a, b)


def test_a_stored_256_thread_choice_is_taken_and_exact(tmp_path, monkeypatch):
    specs = _specs()
    xs = [inputs.make_iq(12, sp, N_SLOTS) for sp in specs]
    path = tmp_path / "tune.tsv"
    monkeypatch.setenv("TT_TUNE_CACHE", str(path))
    _run(specs, xs, autotune=True)                     # writes this device's class keys
    ours, _ = _ours(path)
    path.write_text("".join("\t".join(f[:3] + ["4", "256"]) + "\n" for f in ours))
    wide, geo, _ = _run(specs, xs)
    assert all((g["samples_per_thread"], g["threads_per_cta"], g["samples_per_item"]) == (4, 256, 1024)
               for g in geo)
    monkeypatch.delenv("TT_TUNE_CACHE")
    base, geo_b, _ = _run(specs, xs, engine_kw=dict(samples_per_thread=4))
    assert all(g["threads_per_cta"] == 128 for g in geo_b)
    for sp, x, a, b in zip(specs, xs, wide, base):
        assert np.array_equal(a, b)
        y_ref, q_ref = oracle.run_ue(oracle.OracleUE.from_spec(sp), x)
        assert_int16_close(a, y_ref, q_ref)


def test_a_forced_thread_count_overrides_the_cache(tmp_path, monkeypatch):
    specs = _specs()[:2]
    xs = [inputs.make_iq(13, sp, N_SLOTS) for sp in specs]
    path = tmp_path / "tune.tsv"
    monkeypatch.setenv("TT_TUNE_CACHE", str(path))
    _run(specs, xs, autotune=True)
    ours, _ = _ours(path)
    path.write_text("".join("\t".join(f[:3] + ["4", "256"]) + "\n" for f in ours))
    _, geo, geo_t = _run(specs, xs, autotune=True, engine_kw=dict(threads_per_block=128))
    assert all(g["threads_per_cta"] == 128 for g in geo + geo_t)


def test_an_unwritable_cache_is_reported(tmp_path, monkeypatch):
    specs = _specs()[:2]
    xs = [inputs.make_iq(14, sp, N_SLOTS) for sp in specs]
    monkeypatch.setenv("TT_TUNE_CACHE", str(tmp_path / "no_such_dir" / "tune.tsv"))
    eng = tc.Engine(persistent=True)
    try:
        chans = [tc.Chan(eng, sp, ring_slots=hist_slots(sp) + N_SLOTS + 2) for sp in specs]
        with pytest.raises(tc.TTError) as ei:
            eng.autotune(reps=1)
        assert ei.value.status == tc.TT_ERR_IO
        for ch, x in zip(chans, xs):                   # the engine still runs correctly
            ch.push(0, tc.slots_major(x, ch.n))
        eng.run()
        for sp, ch, x in zip(specs, chans, xs):
            y_ref, q_ref = oracle.run_ue(oracle.OracleUE.from_spec(sp), x)
            assert_int16_close(tc.antenna_major(ch.pull(0, N_SLOTS)), y_ref, q_ref)
    finally:
        eng.close()
