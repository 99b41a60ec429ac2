"""Body of the bounds-checked build's GPU test, run in a child process with TT_CHECKED=1 so that the
binding loads libttchan_checked.so (one library per process).  Prints one JSON line.

1. Parity cases (the six hand-made cases of the parity tests, dense and top-n, several kernel
   geometries) meet the oracle's bars with no out-of-bounds index reported.
2. The tensor-core kernel (BF16, FP16) runs clean within its precision bound.
3. A lowered output bound (test-only TT_TEST_CHECK_SHRINK: the bound is lowered by the whole ring,
   so every output store of the run is out of the shrunk bound) is reported (in the tiled kernel
   exactly one violation per (group of samples, Rx antenna)) with the output-store code, nothing
   is written, the process and GPU stay usable, and the next run on the same engine is correct and
   clean; in both kernels.
"""
import json
import os

import numpy as np

assert os.environ.get("TT_CHECKED") == "1", "run with TT_CHECKED=1"

from paper_2601_08217_gb300 import tt_chan as tc  # noqa: E402
from tests.gpu_harness import hist_slots  # noqa: E402
from tests.helpers import nrmse  # noqa: E402
from tests.test_parity_gpu import CASES, NRMSE_MAX, _case, _oracle, assert_int16_close  # noqa: E402
from tests.test_topn_gpu import _topn_reference  # noqa: E402

TT_CHK_RING_OUT = 11
VARIANTS = [dict(), dict(persistent=True, samples_per_thread=16), dict(threads_per_block=256),
            dict(samples_per_thread=1), dict(persistent=True, samples_per_thread=16, threads_per_block=256)]


def run(spec, x, ns, first, cf32, kw, top_n=0):
    eng = tc.Engine(**kw)
    try:
        ch = tc.Chan(eng, spec, ring_slots=ns + hist_slots(spec) + 1, cf32=cf32, top_n=top_n)
        ch.push(first, x)
        eng.run()
        y = tc.antenna_major(ch.pull(first, ns))
        return y, eng.check_report()
    finally:
        eng.close()


def main():
    assert tc.load()._name.endswith("libttchan_checked.so")
    cases = 0
    for name in CASES:
        spec, x, ns = _case(name)
        y_ref, q_ref = _oracle(spec, x, 5)
        for kw in VARIANTS:
            y, rep = run(spec, x, ns, 5, True, kw)
            assert rep["checked_build"] == 1 and rep["violations"] == 0, (name, kw, rep)
            assert nrmse(y, y_ref) <= NRMSE_MAX, (name, kw)
            q, rep = run(spec, x, ns, 5, False, kw)
            assert rep["violations"] == 0, (name, kw, rep)
            assert_int16_close(q, y_ref, q_ref)
            cases += 2
    for name, top_n in (("mimo22_noise", 3), ("nr20mhz_mimo_1ms_trace", 4)):
        spec, x, ns = _case(name)
        for kw in (dict(persistent=True), dict(persistent=True, threads_per_block=256)):
            q, rep = run(spec, x, ns, 0, False, kw, top_n=top_n)
            assert rep["violations"] == 0, (name, kw, rep)
            y_ref, q_ref, _ = _topn_reference(spec, x, top_n, q, cf32=False)
            assert_int16_close(q, y_ref, q_ref)
            cases += 1

    # the tensor-core kernel (BF16 and FP16) on the multi-antenna cases, within the precision bound
    from paper_2601_08217_gb300 import inputs
    for prec in (tc.TT_BF16_TC, tc.TT_FP16_TC):
        sp = inputs.make_ue(31, 0, 1024, 40, 120, 100.0, 4, n_tx=2, n_rx=2)
        x = inputs.make_iq(31, sp, 2)
        y_ref, _ = _oracle(sp, x, 0)
        eng = tc.Engine()
        try:
            ch = tc.Chan(eng, sp, ring_slots=4, cf32=True, precision=prec)
            ch.push(0, x)
            eng.run()
            y = tc.antenna_major(ch.pull(0, 2))
            rep = eng.check_report()
        finally:
            eng.close()
        assert rep["violations"] == 0, (prec, rep)
        assert 20 * np.log10(nrmse(y, y_ref)) < -40.0, prec
        cases += 1

    # planted: every output store of one run falls outside the lowered bound
    spec, x, ns = _case("mimo22_noise")
    y_ref, q_ref = _oracle(spec, x, 0)
    n = spec.n
    eng = tc.Engine()
    try:
        q_slots = ns + hist_slots(spec) + 1
        ch = tc.Chan(eng, spec, ring_slots=q_slots)
        xs = tc.slots_major(x, n)
        os.environ["TT_TEST_CHECK_SHRINK"] = str(q_slots * spec.n_rx * n)
        try:
            ch.push(0, xs[:1])
            eng.run()
            eng.sync()
        finally:
            del os.environ["TT_TEST_CHECK_SHRINK"]
        planted = eng.check_report()
        groups = n // ch.geometry()["samples_per_thread"]
        assert planted["violations"] == groups * spec.n_rx, (planted, groups)
        assert planted["first_code"] == TT_CHK_RING_OUT
        ch.pull(0, 1)                                   # slot 0 was not written
        ch.push(1, xs[1:ns])
        eng.run()
        q = tc.antenna_major(ch.pull(1, ns - 1))
        after = eng.check_report()
        assert after["violations"] == 0, after
        assert_int16_close(q, y_ref[:, n:], q_ref[:, n:])
    finally:
        eng.close()
    # the same in the tensor-core kernel: reported, nothing written, the next run correct
    sp = inputs.make_ue(31, 1, 1024, 24, 100, 100.0, 5, n_tx=2, n_rx=2)
    x = tc.slots_major(inputs.make_iq(32, sp, 3), sp.n)
    y_ref, _ = _oracle(sp, inputs.make_iq(32, sp, 3), 0)
    eng = tc.Engine()
    try:
        ch = tc.Chan(eng, sp, ring_slots=5, cf32=True, precision=tc.TT_BF16_TC)
        os.environ["TT_TEST_CHECK_SHRINK"] = str(5 * sp.n_rx * sp.n)
        try:
            ch.push(0, x[:1])
            eng.run()
            eng.sync()
        finally:
            del os.environ["TT_TEST_CHECK_SHRINK"]
        tc_planted = eng.check_report()
        assert tc_planted["violations"] > 0 and tc_planted["first_code"] == TT_CHK_RING_OUT, tc_planted
        ch.pull(0, 1)
        ch.push(1, x[1:3])
        eng.run()
        y = tc.antenna_major(ch.pull(1, 2))
        assert eng.check_report()["violations"] == 0
        assert 20 * np.log10(nrmse(y, y_ref[:, sp.n:])) < -40.0
    finally:
        eng.close()
    print(json.dumps({"cases": cases, "planted": planted, "groups": groups, "after": after, "tc_planted": tc_planted}))


if __name__ == "__main__":
    main()
