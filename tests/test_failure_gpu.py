"""Failure detection on the GPU without a fault: the tensor-core kernel's bounded waits.

With the test-only switch TT_TEST_TC_NO_MMA=1 set at a run, the kernel's MMA warp issues no MMA and
no commit.  Nothing is then in flight on the tensor core, and the builders' waits for ring slots and
accumulators run out (about a second).  The kernel records the expiry in the engine's status word,
frees its tensor memory and exits; tt_engine_sync reports TT_ERR_TIMEOUT and clears the word.  The
next run on the same engine, with the switch unset, must be correct.  A leaked tensor-memory
allocation would make that run's kernel wait forever in tcgen05.alloc, so it would not complete.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.helpers import nrmse

pytestmark = pytest.mark.gpu


def test_tensor_core_wait_expiry_is_reported_and_the_engine_recovers():
    sp = inputs.make_ue(4, 0, 1024, 16, 60, 100.0, 4, n_tx=2, n_rx=2)
    x = inputs.make_iq(4, sp, 2)
    y_ref, _ = oracle.run_ue(oracle.OracleUE.from_spec(sp), x)
    eng = tc.Engine(form="batched")
    try:
        ch = tc.Chan(eng, sp, ring_slots=4, cf32=True, precision=tc.TT_BF16_TC)
        slots = tc.slots_major(x, sp.n)
        ch.push(0, slots[0:1])
        os.environ["TT_TEST_TC_NO_MMA"] = "1"
        try:
            eng.run()
        finally:
            del os.environ["TT_TEST_TC_NO_MMA"]
        with pytest.raises(tc.TTError) as ei:
            eng.sync()
        assert ei.value.status == tc.TT_ERR_TIMEOUT
        assert "bounded wait" in str(ei.value)
        eng.sync()                                   # the status word was cleared
        ch.push(1, slots[1:2])
        eng.run()
        eng.sync()
        y = tc.antenna_major(ch.pull(0, 2))          # slot 0 is invalid, slot 1 must be right
        n = sp.n
        assert 20 * np.log10(nrmse(y[:, n:], y_ref[:, n:])) < -40.0   # BF16 bound of the precision tests
    finally:
        eng.close()
