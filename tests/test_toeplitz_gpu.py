"""Block-Toeplitz tensor-core form (tcgen05, BF16/FP16 operands, FP32 accumulation).

Pin: taps and inputs exactly representable in BF16 (and FP16) with static
taps make every product and partial sum exact, so the tensor-core output must
equal the FP32 path's and the oracle's bit for bit; this fixes the operand
layouts (descriptor strides, polyphase indexing, Toeplitz signs).  Random
channels are then checked against the FP64 oracle by EVM, stated per
precision, pre- and post-packing."""
import numpy as np
import pytest

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.gpu_harness import run_gpu
from tests.helpers import nrmse

pytestmark = pytest.mark.gpu


class Spec:
    def __init__(self, L, n_tx, n_rx, delays, taps, noise_var=0.0, loop=True, seed=5, ue_id=0):
        self.symbol_len = list(L)
        self.n_tx, self.n_rx = n_tx, n_rx
        self.delays = np.asarray(delays, dtype=np.int32)
        self.taps = np.asarray(taps, dtype=np.complex64)
        self.step_samples, self.loop = 0.0, loop
        self.noise_var, self.seed, self.ue_id = noise_var, seed, ue_id
        self.max_delay = int(self.delays.max())

    @property
    def n(self):
        return int(sum(self.symbol_len))


def evm_db(y, ref):
    return 20 * np.log10(nrmse(y, ref))


@pytest.mark.parametrize("prec", [tc.TT_BF16_TC, tc.TT_FP16_TC])
@pytest.mark.parametrize("n_ant,K,n_fft", [(4, 96, 1024), (1, 24, 1024), (2, 128, 1024), (3, 40, 4096)])
def test_exactly_representable_inputs_give_exact_output(prec, n_ant, K, n_fft):
    rng = np.random.default_rng(40 + K)
    L = inputs.nr_symbol_lengths(n_fft)                   # 20 MHz: one tile group; 100 MHz: two per symbol
    d = np.arange(K) if K <= 96 else np.sort(rng.choice(np.arange(128), K, replace=False))
    h = (rng.integers(-8, 9, size=(1, n_ant, n_ant, K)) + 1j * rng.integers(-8, 9, size=(1, n_ant, n_ant, K))) / 8
    taps = np.repeat(h, 3, axis=0).astype(np.complex64)  # static: H[a+1] - H[a] = 0
    spec = Spec(L, n_ant, n_ant, d, taps)
    x = rng.integers(-127, 128, size=(n_ant, 2 * spec.n, 2)).astype(np.int16)
    y_ref, q_ref = oracle.run_ue(oracle.OracleUE.from_spec(spec), x)
    y_tc = run_gpu([spec], [x], 2, cf32=True, precision=prec)[0]
    y_fp = run_gpu([spec], [x], 2, cf32=True)[0]
    assert np.array_equal(y_fp.astype(np.complex128), y_ref)
    assert np.array_equal(y_tc.astype(np.complex128), y_ref)
    q_tc = run_gpu([spec], [x], 2, cf32=False, precision=prec)[0]
    assert np.array_equal(q_tc, q_ref)


def test_time_varying_exact_taps_match_fp32_closely():
    """Exact operands but interpolated taps: A + tau*B vs the per-tap interpolation differ only by FP32 rounding."""
    rng = np.random.default_rng(3)
    L = inputs.nr_symbol_lengths(1024)
    K = 64
    h = (rng.integers(-8, 9, size=(4, 2, 2, K)) + 1j * rng.integers(-8, 9, size=(4, 2, 2, K))) / 8
    spec = Spec(L, 2, 2, np.arange(K), h.astype(np.complex64))
    x = rng.integers(-127, 128, size=(2, 2 * spec.n, 2)).astype(np.int16)
    y_ref, _ = oracle.run_ue(oracle.OracleUE.from_spec(spec), x)
    y_tc = run_gpu([spec], [x], 2, cf32=True, precision=tc.TT_BF16_TC)[0]
    assert nrmse(y_tc, y_ref) < 1e-6


@pytest.mark.parametrize("prec,bound_db", [(tc.TT_BF16_TC, -40.0), (tc.TT_FP16_TC, -55.0)])
def test_dense_4x4_96tap_evm_against_oracle(prec, bound_db):
    specs = inputs.workload_precision(n_ues=2, n_slots_trace=2)
    for sp in specs:
        sp.noise_var = 0.0
    xs = [inputs.make_iq(4, sp, 2) for sp in specs]
    ys = run_gpu(specs, xs, 2, cf32=True, precision=prec)
    qs = run_gpu(specs, xs, 2, cf32=False, precision=prec)
    for sp, x, y, q in zip(specs, xs, ys, qs):
        y_ref, _ = oracle.run_ue(oracle.OracleUE.from_spec(sp), x)
        pre = evm_db(y, y_ref)
        post = evm_db(q[..., 0] + 1j * q[..., 1], y_ref)
        print(f"precision {prec}: EVM pre-pack {pre:.1f} dB, post-pack {post:.1f} dB")
        assert pre < bound_db and post < bound_db


def test_tensor_core_and_fp32_channels_in_one_engine():
    specs = inputs.workload_precision(n_ues=2, n_slots_trace=2) + inputs.workload_plain_16ue(2, n_ues=2)
    xs = [inputs.make_iq(4, sp, 2) for sp in specs]
    eng = tc.Engine()
    chans = [tc.Chan(eng, sp, ring_slots=4, cf32=True, precision=(tc.TT_FP16_TC if i < 2 else tc.TT_FP32))
             for i, sp in enumerate(specs)]
    for ch, x in zip(chans, xs):
        ch.push(0, x)
    eng.run()
    mixed = [tc.antenna_major(ch.pull(0, 2)) for ch in chans]
    eng.close()
    alone_tc = run_gpu(specs[:2], xs[:2], 2, cf32=True, precision=tc.TT_FP16_TC)
    alone_fp = run_gpu(specs[2:], xs[2:], 2, cf32=True)
    for a, b in zip(mixed, alone_tc + alone_fp):
        assert np.array_equal(a, b)


_FULL = {}


def _full_size_refs():
    """The whole precision workload (64 UEs, 4x4, 96 taps, 100 MHz), one slot, AWGN off; oracle once."""
    if not _FULL:
        specs = inputs.workload_precision(n_ues=64, n_slots_trace=2)
        for sp in specs:
            sp.noise_var = 0.0
        xs = [inputs.make_iq(4, sp, 1) for sp in specs]
        _FULL["specs"], _FULL["xs"] = specs, xs
        _FULL["refs"] = [oracle.run_ue(oracle.OracleUE.from_spec(sp), x)[0] for sp, x in zip(specs, xs)]
    return _FULL["specs"], _FULL["xs"], _FULL["refs"]


@pytest.mark.parametrize("prec,bound_db", [(tc.TT_BF16_TC, -40.0), (tc.TT_FP16_TC, -55.0)])
def test_full_size_64_ues_evm_against_oracle(prec, bound_db):
    """Every UE of the precision workload, one slot in one launch: the EVM bound holds for each."""
    specs, xs, refs = _full_size_refs()
    ys = run_gpu(specs, xs, 1, cf32=True, precision=prec)
    worst = max(evm_db(y, y_ref) for y, y_ref in zip(ys, refs))
    print(f"precision {prec}: worst EVM over 64 UEs {worst:.1f} dB")
    assert worst < bound_db


@pytest.mark.parametrize("prec", [tc.TT_BF16_TC, tc.TT_FP16_TC])
def test_fused_awgn_equals_the_fp32_path(prec):
    """Exact operands, static taps and AWGN on (4x4, 96 taps, 100 MHz: three groups per symbol): the
    tensor-core sums are exact and its epilogue adds the same Philox noise to them, so the output
    equals the FP32 path's bit for bit, and the oracle's within the FP32 tolerance."""
    rng = np.random.default_rng(77)
    L = inputs.nr_symbol_lengths(4096)
    K = 96
    h = (rng.integers(-8, 9, size=(1, 4, 4, K)) + 1j * rng.integers(-8, 9, size=(1, 4, 4, K))) / 8
    spec = Spec(L, 4, 4, np.arange(K), np.repeat(h, 3, axis=0), noise_var=inputs.noise_var_for_snr(20.0),
                ue_id=5)
    x = rng.integers(-127, 128, size=(4, 2 * spec.n, 2)).astype(np.int16)
    y_fp = run_gpu([spec], [x], 2, cf32=True)[0]
    y_tc = run_gpu([spec], [x], 2, cf32=True, precision=prec)[0]
    assert np.array_equal(y_tc, y_fp)
    y_ref, _ = oracle.run_ue(oracle.OracleUE.from_spec(spec), x)
    assert np.std(y_ref) > 50 and nrmse(y_tc, y_ref) <= 1e-5
