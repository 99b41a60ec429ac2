"""Sparse convolution (Sec. III-C: only the top-n dominant taps of each time step) on the GPU,
through the C ABI, against the FP64 oracle's top-n mode.

The kernel and the oracle take the tap selection in the same precision (binary32 powers,
p = fma(re, re, im * im), ties to the lower tap index), so the kept sets agree; the bars are
those of the dense path: FP32 pre-pack NRMSE <= 1e-5, int16 within +-1 LSB at rounding ties,
bit-exact where every operation is exact.
"""
import numpy as np
import pytest

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.gpu_harness import run_gpu
from tests.helpers import nrmse
from tests.test_parity_gpu import Spec, _case, assert_int16_close

pytestmark = pytest.mark.gpu

NRMSE_MAX = 1e-5


def _oracle_topn(spec, x, top_n, first_slot=0):
    return oracle.run_ue(oracle.OracleUE.from_spec(spec, top_n=top_n), x, s_first=first_slot)


TOPN_CASES = [("siso_odd_lengths", 2), ("delay_beyond_slot", 1), ("mimo22_noise", 3),
              ("mimo_4tx_3rx_tracetime", 5), ("nr5mhz_loop_noise", 6), ("nr20mhz_mimo_1ms_trace", 4)]


@pytest.mark.parametrize("spt", [0, 1, 2, 16])
@pytest.mark.parametrize("case,top_n", TOPN_CASES)
def test_top_n_matches_oracle(case, top_n, spt):
    spec, x, ns = _case(case)
    y_ref, q_ref = _oracle_topn(spec, x, top_n)
    y_full, _ = _oracle_topn(spec, x, 0)
    assert nrmse(y_ref, y_full) > 1e-3                  # the sparse result differs from all taps
    y = run_gpu([spec], [x], ns, cf32=True, spt=spt, persistent=True, top_n=top_n)[0]
    assert nrmse(y, y_ref) <= NRMSE_MAX
    q = run_gpu([spec], [x], ns, spt=spt, persistent=True, top_n=top_n)[0]
    assert_int16_close(q, y_ref, q_ref)


def test_top_n_at_or_above_tap_count_is_the_dense_path():
    spec, x, ns = _case("mimo22_noise")
    K = len(spec.delays)
    dense = run_gpu([spec], [x], ns)[0]
    for n in (K, K + 5):
        assert np.array_equal(run_gpu([spec], [x], ns, top_n=n)[0], dense)


def test_top_n_ties_and_switching_are_bit_exact():
    """Small integer taps and inputs: every FP32 operation is exact, so the GPU must equal the
    oracle bit for bit, with ties broken toward the lower tap and the kept set switching
    between symbols (the dominant tap moves from anchor to anchor)."""
    rng = np.random.default_rng(41)
    L = [16, 16, 16, 16]
    d = [0, 1, 4, 9, 17, 30]
    T = 4 * 3 + 1
    mag = rng.integers(1, 3, size=(T, 1, 1, len(d)))          # powers 1 or 4: many ties
    taps = (mag * rng.choice([1, -1, 1j, -1j], size=mag.shape)).astype(np.complex64)
    spec = Spec(L, 1, 1, d, taps)
    x = rng.integers(-300, 300, size=(1, 3 * 64, 2)).astype(np.int16)
    for top_n in (1, 2, 4):
        _, q_ref = _oracle_topn(spec, x, top_n)
        # interpolation by tau = m / 16 of integer taps is exact in FP32; the sums stay integral * 2^-4
        q = run_gpu([spec], [x], 3, top_n=top_n)[0]
        assert np.array_equal(q, q_ref)


def test_sparse_and_dense_channels_share_a_launch():
    """Channels with and without top-n in one engine run: each equals its own run alone."""
    specs = inputs.workload_plain_16ue(n_slots=4, n_ues=4)
    xs = [inputs.make_iq(2, sp, 3) for sp in specs]
    tops = [0, 8, 0, 3]
    mixed = run_gpu(specs, xs, 3, top_n=tops, persistent=True)
    for sp, x, t, m in zip(specs, xs, tops, mixed):
        alone = run_gpu([sp], [x], 3, top_n=t, persistent=True)[0]
        assert np.array_equal(m, alone)
    y_ref, q_ref = _oracle_topn(specs[3], xs[3], 3)
    assert_int16_close(mixed[3], y_ref, q_ref)


def test_top_n_is_refused_outside_the_fp32_batched_form():
    spec, _, _ = _case("siso_odd_lengths")
    for form, prec in (("plain", tc.TT_FP32), ("batched", tc.TT_BF16_TC)):
        eng = tc.Engine(form=form)
        try:
            with pytest.raises(tc.TTError) as ex:
                tc.Chan(eng, spec, precision=prec, top_n=2)
            assert ex.value.status == tc.TT_ERR_INVALID
        finally:
            eng.close()


@pytest.mark.parametrize("spt", [8, 16])
def test_top_n_on_the_40mhz_siso_workload(spt):
    """Top 8 of 24 taps on two UEs of the 40 MHz benchmark workload, at 8 and 16 samples per thread
    (the single-antenna variants with bounded registers), against the oracle's top-n mode."""
    specs = inputs.workload_plain_16ue(3, n_ues=2)
    for sp in specs:
        x = inputs.make_iq(2, sp, 3)
        y_ref, q_ref = _oracle_topn(sp, x, 8)
        y = run_gpu([sp], [x], 3, cf32=True, spt=spt, persistent=True, top_n=8)[0]
        assert nrmse(y, y_ref) <= NRMSE_MAX
        q = run_gpu([sp], [x], 3, spt=spt, persistent=True, top_n=8)[0]
        assert_int16_close(q, y_ref, q_ref)
