"""Sparse convolution (Sec. III-C: only the top-n dominant taps of each time step) on the GPU,
through the C ABI, against the FP64 oracle's top-n mode.

The oracle ranks the taps by their FP64 power.  The kernel ranks them in binary32, so where two
powers lie within binary32 rounding of each other at the n-th place, either tap is a correct
choice.  The check therefore starts from the oracle's FP64 selection and, only for symbols whose
output differs from the GPU's, tries the other valid selections of that anchor (those that swap
near-tied taps, `tests.helpers.topn_selections`), re-running the oracle with each.  The bars are
those of the dense path: FP32 pre-pack NRMSE <= 1e-5, int16 within +-1 LSB at rounding ties,
bit-exact where every operation is exact.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.gpu_harness import run_gpu
from tests.helpers import nrmse, topn_selections
from tests.test_parity_gpu import Spec, _case, assert_int16_close

pytestmark = pytest.mark.gpu

NRMSE_MAX = 1e-5


def _oracle_topn(spec, x, top_n, first_slot=0):
    return oracle.run_ue(oracle.OracleUE.from_spec(spec, top_n=top_n), x, s_first=first_slot)


def _topn_reference(spec, x, top_n, out, cf32, first_slot=0):
    """The oracle's (y, q) for the selection the GPU made, provided that selection is valid, and the
    number of symbols where it differs from the FP64 selection.  out is the GPU's output
    (complex [n_rx][n_slots*N] if cf32, else int16 [n_rx][n_slots*N][2])."""
    ue = oracle.OracleUE.from_spec(spec, top_n=top_n)
    L = list(spec.symbol_len)
    nsym, n = len(L), spec.n
    ns = x.shape[1] // n
    starts = np.concatenate([[0], np.cumsum(L)[:-1]]).astype(int)
    sels = [topn_selections(oracle.anchor(ue, first_slot * nsym + i), top_n) for i in range(ns * nsym + 1)]
    mask = np.stack([b for b, _ in sels])
    y_ref, q_ref = oracle.run_ue(ue, x, s_first=first_slot, keep=mask)
    y_fp64, _ = _oracle_topn(spec, x, top_n, first_slot)
    assert nrmse(y_ref, y_fp64) == 0.0                 # the base selection is the oracle's own

    def err(rng, yr, qr):
        if cf32:
            return nrmse(out[:, rng], yr[:, rng])
        return int(np.abs(out[:, rng].astype(np.int32) - qr[:, rng].astype(np.int32)).max())

    bar = NRMSE_MAX if cf32 else 1
    changed = 0
    for i in range(ns * nsym):
        alts = sels[i][1]
        sl, j = divmod(i, nsym)
        rng = slice(sl * n + starts[j], sl * n + starts[j] + L[j])
        if not alts or err(rng, y_ref, q_ref) <= bar:
            continue
        links = list(alts)
        best = None
        for combo in itertools.islice(itertools.product(*[alts[k] for k in links]), 256):
            m = mask.copy()
            for (r, t), sel in zip(links, combo):
                m[i, r, t] = sel
            yr, qr = oracle.run_ue(ue, x, s_first=first_slot, keep=m)
            e = err(rng, yr, qr)
            if best is None or e < best[0]:
                best = (e, m, yr, qr)
        if best[0] < err(rng, y_ref, q_ref):
            _, mask, y_ref, q_ref = best
            changed += 1
    return y_ref, q_ref, changed


def _check_topn(spec, x, ns, top_n, spt=0, persistent=True, tpb=0):
    y = run_gpu([spec], [x], ns, cf32=True, spt=spt, persistent=persistent, top_n=top_n, tpb=tpb)[0]
    y_ref, _, changed_y = _topn_reference(spec, x, top_n, y, cf32=True)
    assert nrmse(y, y_ref) <= NRMSE_MAX
    q = run_gpu([spec], [x], ns, spt=spt, persistent=persistent, top_n=top_n, tpb=tpb)[0]
    y_ref, q_ref, changed_q = _topn_reference(spec, x, top_n, q, cf32=False)
    assert_int16_close(q, y_ref, q_ref)
    return changed_y, changed_q


TOPN_CASES = [("siso_odd_lengths", 2), ("delay_beyond_slot", 1), ("mimo22_noise", 3),
              ("mimo_4tx_3rx_tracetime", 5), ("nr5mhz_loop_noise", 6), ("nr20mhz_mimo_1ms_trace", 4)]


@pytest.mark.parametrize("spt,tpb", [(0, 0), (1, 0), (2, 0), (16, 0), (0, 256), (16, 256)])
@pytest.mark.parametrize("case,top_n", TOPN_CASES)
def test_top_n_matches_oracle(case, top_n, spt, tpb):
    spec, x, ns = _case(case)
    y_ref, _ = _oracle_topn(spec, x, top_n)
    y_full, _ = _oracle_topn(spec, x, 0)
    assert nrmse(y_ref, y_full) > 1e-3                  # the sparse result differs from all taps
    _check_topn(spec, x, ns, top_n, spt=spt, tpb=tpb)


def test_near_tie_accepts_the_binary32_choice():
    """Taps 0 and 1 have FP64 powers 1 and 1 + 2^-24 (tap 1 is 1 + 2^-12 i).  The oracle keeps tap 1.
    In binary32, fma(1, 1, 2^-24) rounds to 1 (the midpoint goes to even), the two powers tie and the
    lower index, tap 0, is kept.  Both selections are valid; the check must find the GPU's and match
    the oracle re-run with it."""
    rng = np.random.default_rng(77)
    L = [16, 16, 16, 16]
    d = [0, 3, 7, 12]
    prof = np.array([1.0, 1.0 + 2.0 ** -12 * 1j, 0.25, 0.1j], dtype=np.complex64)
    assert prof[1].imag == 2.0 ** -12
    taps = np.tile(prof.reshape(1, 1, 1, 4), (4 * 2 + 1, 1, 1, 1))
    spec = Spec(L, 1, 1, d, taps)
    x = rng.integers(-3000, 3000, size=(1, 2 * 64, 2)).astype(np.int16)
    changed_y, changed_q = _check_topn(spec, x, 2, 1)
    assert changed_y == 8 and changed_q == 8            # every symbol took the other valid choice


def test_top_n_at_or_above_tap_count_is_the_dense_path():
    spec, x, ns = _case("mimo22_noise")
    K = len(spec.delays)
    dense = run_gpu([spec], [x], ns)[0]
    for n in (K, K + 5):
        assert np.array_equal(run_gpu([spec], [x], ns, top_n=n)[0], dense)


def test_top_n_ties_and_switching_are_bit_exact():
    """Small integer taps and inputs: every FP32 operation is exact, so the GPU must equal the
    oracle bit for bit, with ties broken toward the lower tap and the kept set switching
    between symbols (the dominant tap moves from anchor to anchor).  Powers of 1 and 4 are exact
    in binary32 and FP64 alike, so both rankings see the same ties and the FP64 selection is the
    only one accepted here."""
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
    y_ref, q_ref, _ = _topn_reference(specs[3], xs[3], 3, mixed[3], cf32=False)
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
        _check_topn(sp, x, 3, 8, spt=spt)
