"""Uplink aggregation at a cell (Sec. III-A: the gNB convolves each UE's uplink stream and
aggregates them) on the GPU, through the C ABI, against the oracle's run_cell.

Bars: complex64 cell output within NRMSE 1e-5 of the oracle (the members' FP32 convolutions and
an FP32 sum in member order); int16 cell output within +-1 LSB at rounding ties or saturation.
"""
import numpy as np
import pytest

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.helpers import nrmse
from tests.test_parity_gpu import assert_int16_close

pytestmark = pytest.mark.gpu


def _members(n_ues, n_slots, n_rx=1, n_tx=(1,), seed_base=0):
    """Cell members: the 40 MHz 24-tap UEs, noise off (the cell carries the noise)."""
    specs = inputs.workload_plain_16ue(n_slots=n_slots + 1, n_ues=n_ues)
    out = []
    for i, sp in enumerate(specs):
        sp.noise_var = 0.0
        if n_rx != 1 or n_tx != (1,):
            nt = n_tx[i % len(n_tx)]
            rng = np.random.default_rng(seed_base + i)
            T = sp.taps.shape[0]
            z = rng.standard_normal((T, n_rx, nt, len(sp.delays))) + 1j * rng.standard_normal((T, n_rx, nt, len(sp.delays)))
            sp.taps = (z / np.sqrt(2 * len(sp.delays) * nt)).astype(np.complex64)
            sp.n_tx, sp.n_rx = nt, n_rx
        out.append(sp)
    return out


def _run_cell_gpu(specs, xs, n_slots, cell_kw, cf32=False, precisions=None, stream=False):
    eng = tc.Engine(persistent=True)
    try:
        cell = tc.Cell(eng, samples_per_slot=specs[0].n, n_rx=specs[0].n_rx, cf32=cf32,
                       ring_slots=(2 if stream else n_slots), **cell_kw)
        chans = []
        for i, sp in enumerate(specs):
            prec = precisions[i] if precisions else tc.TT_FP32
            ch = tc.Chan(eng, sp, ring_slots=(3 if stream else n_slots + 2), cf32=True, precision=prec)
            cell.attach(ch)
            chans.append(ch)
        if stream:
            outs = []
            for s in range(n_slots):
                for ch, x in zip(chans, xs):
                    ch.push(s, tc.slots_major(x, ch.n)[s:s + 1])
                eng.run()
                outs.append(cell.pull(s, 1))
            y = np.concatenate(outs, axis=0)
        else:
            for ch, x in zip(chans, xs):
                ch.push(0, x)
            eng.run()
            y = cell.pull(0, n_slots)
        return tc.antenna_major(y)
    finally:
        eng.close()


def _oracle_cell(specs, xs, seed, cell_id, noise_var):
    ues = [oracle.OracleUE.from_spec(sp) for sp in specs]
    return oracle.run_cell(ues, xs, seed=seed, cell_id=cell_id, noise_var=noise_var)


CELL = dict(cell_id=7, seed=0x5EED, noise_var=inputs.noise_var_for_snr(20.0))


def test_cell_of_siso_ues_matches_oracle():
    specs = _members(6, 3)
    xs = [inputs.make_iq(2, sp, 3) for sp in specs]
    y_ref, q_ref = _oracle_cell(specs, xs, CELL["seed"], CELL["cell_id"], CELL["noise_var"])
    y = _run_cell_gpu(specs, xs, 3, CELL, cf32=True)
    assert nrmse(y, y_ref) <= 1e-5
    q = _run_cell_gpu(specs, xs, 3, CELL)
    assert_int16_close(q, y_ref, q_ref)


def test_cell_of_mimo_ues_with_mixed_tx_counts():
    specs = _members(4, 2, n_rx=2, n_tx=(1, 2), seed_base=90)
    xs = [inputs.make_iq(2, sp, 2) for sp in specs]
    y_ref, q_ref = _oracle_cell(specs, xs, 11, 3, 0.0)
    y = _run_cell_gpu(specs, xs, 2, dict(cell_id=3, seed=11, noise_var=0.0), cf32=True)
    assert nrmse(y, y_ref) <= 1e-5
    q = _run_cell_gpu(specs, xs, 2, dict(cell_id=3, seed=11, noise_var=0.0))
    assert_int16_close(q, y_ref, q_ref)


def test_cell_streamed_through_small_rings_equals_bulk():
    specs = _members(3, 5)
    xs = [inputs.make_iq(2, sp, 5) for sp in specs]
    bulk = _run_cell_gpu(specs, xs, 5, CELL)
    streamed = _run_cell_gpu(specs, xs, 5, CELL, stream=True)
    assert np.array_equal(bulk, streamed)


def test_cell_with_a_tensor_core_member():
    """Members may run either form; a BF16 tensor-core member keeps the cell close to the oracle
    (its EVM bound), the FP32 members exact to FP32 rounding."""
    rng = np.random.default_rng(5)
    specs = inputs.workload_precision(n_ues=2, n_slots_trace=2)
    for sp in specs:
        sp.noise_var = 0.0
    xs = [inputs.make_iq(4, sp, 1) for sp in specs]
    y_ref, _ = _oracle_cell(specs, xs, 1, 1, 0.0)
    y = _run_cell_gpu(specs, xs, 1, dict(cell_id=1, seed=1, noise_var=0.0), cf32=True,
                      precisions=[tc.TT_FP32, tc.TT_BF16_TC])
    evm = 20 * np.log10(np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref))
    assert evm < -40.0


def test_cell_refusals():
    specs = _members(2, 2)
    eng = tc.Engine()
    try:
        cell = tc.Cell(eng, cell_id=0, samples_per_slot=specs[0].n)
        int16_chan = tc.Chan(eng, specs[0])                        # packed output: refused
        with pytest.raises(tc.TTError) as ex:
            cell.attach(int16_chan)
        assert ex.value.status == tc.TT_ERR_INVALID
        noisy = inputs.workload_plain_16ue(n_slots=3, n_ues=1)[0]   # own noise: refused
        with pytest.raises(tc.TTError) as ex:
            cell.attach(tc.Chan(eng, noisy, cf32=True))
        assert ex.value.status == tc.TT_ERR_INVALID
        with pytest.raises(tc.TTError) as ex:                       # odd N
            tc.Cell(eng, cell_id=1, samples_per_slot=1001)
        assert ex.value.status == tc.TT_ERR_INVALID
        m = tc.Chan(eng, specs[1], cf32=True, ring_slots=4)
        cell.attach(m)
        with pytest.raises(tc.TTError) as ex:                       # attached twice
            cell.attach(m)
        assert ex.value.status == tc.TT_ERR_STATE
        m.push(0, inputs.make_iq(2, specs[1], 1))
        eng.run()
        with pytest.raises(tc.TTError) as ex:                       # the member's output is the cell's
            m.pull(0, 1)
        assert ex.value.status == tc.TT_ERR_STATE
        with pytest.raises(tc.TTError) as ex:                       # a member outlives no cell
            tc.tt_chan_destroy(m.h)
        assert ex.value.status == tc.TT_ERR_STATE
        late = tc.Chan(eng, specs[0], cf32=True)
        late.spec.noise_var = 0.0
        with pytest.raises(tc.TTError) as ex:                       # the cell has started
            cell.attach(late)
        assert ex.value.status in (tc.TT_ERR_STATE, tc.TT_ERR_INVALID)
        assert cell.pull(0, 1).shape == (1, 1, specs[0].n, 2)
        cell.destroy()
    finally:
        eng.close()


def test_cell_members_served_by_the_request_loop():
    """The serving loop admits cell members like any channel and drains the cell ring: the
    aggregation keeps consuming the members' outputs, so requests keep completing (independent
    arrivals let members drift apart, so some are refused when one runs a ring ahead)."""
    specs = _members(4, 3)
    eng = tc.Engine(persistent=True)
    try:
        cell = tc.Cell(eng, cell_id=5, samples_per_slot=specs[0].n, ring_slots=4)
        for sp in specs:
            ch = tc.Chan(eng, sp, cf32=True, ring_slots=8)
            cell.attach(ch)
        rep = tc.tt_engine_serve(eng.h, duration_s=0.2, warmup_s=0.02, slot_period_us=500.0, jitter_us=50.0,
                                 deadline_us=500.0, seed=3, release_outputs=True)
        assert rep["completed"] > 0.5 * rep["requests"]
    finally:
        eng.close()
