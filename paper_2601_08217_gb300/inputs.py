"""Seeded synthetic inputs for the per-UE channel-convolution path.

This module draws the data that both the FP64 oracle and the CUDA path consume:
complex int16 IQ slot buffers, integer tap delays, power-delay profiles, and
time-varying complex tap anchors (the "channel traces" of Sec. IV, which the
paper replays from files built from 3GPP PDPs with Jakes Doppler, ray tracing
or measurements).  None of those trace sources are available, so a seeded
sum-of-sinusoids Rayleigh generator stands in for them.

It holds none of the method's arithmetic: no convolution, no tap
interpolation, no noise, no packing.  Everything here is an input.

Seeding: every array is drawn from
``numpy.random.default_rng(SeedSequence([0x77170000 + workload, ue, antenna, stream]))``
so any UE of any workload can be regenerated alone.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

SEED_BASE = 0x7717_0000
IQ_STD = 1024.0            # 2^10 per component
P_X_NOMINAL = 2.0 * IQ_STD ** 2   # nominal complex input power used to set the noise level

# stream ids inside one SeedSequence family
_S_IQ, _S_DELAY, _S_TRACE = 0, 1, 2


def rng_for(workload: int, ue: int, antenna: int = 0, stream: int = 0) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([SEED_BASE + workload, ue, antenna, stream]))


# ----------------------------------------------------------------------------
# NR numerology (30 kHz SCS, normal cyclic prefix, 14 symbols per 0.5 ms slot)
# ----------------------------------------------------------------------------
def nr_symbol_lengths(n_fft: int) -> List[int]:
    """Symbol lengths (CP + FFT) in samples for one 30 kHz slot.

    The first symbol of each half-subframe carries the long CP: with
    B = n_fft/128 it is 139*B samples long and the other 13 are 137*B.
    """
    if n_fft % 128:
        raise ValueError("n_fft must be a multiple of 128")
    b = n_fft // 128
    return [139 * b] + [137 * b] * 13


BANDWIDTH_NFFT = {5: 256, 20: 1024, 40: 2048, 100: 4096}   # MHz -> FFT size at 30 kHz


def sample_rate(n_fft: int) -> float:
    return n_fft * 30e3


def anchor_starts(n_anchors: int, symbol_len: Sequence[int]) -> np.ndarray:
    """Start sample of every symbol a = 0..n_anchors-1 (slot-periodic numerology)."""
    L = np.asarray(symbol_len, dtype=np.int64)
    n = int(L.sum())
    starts = np.concatenate([[0], np.cumsum(L)[:-1]])
    a = np.arange(n_anchors, dtype=np.int64)
    return (a // len(L)) * n + starts[a % len(L)]


# ----------------------------------------------------------------------------
# IQ, delays, profiles
# ----------------------------------------------------------------------------
def gen_iq(rng: np.random.Generator, n_ant: int, n_samples: int, std: float = IQ_STD) -> np.ndarray:
    """Gaussian complex IQ, std ``std`` per component, rounded and clipped to int16.

    Returns int16 array [n_ant, n_samples, 2] (I, Q interleaved).
    """
    v = rng.standard_normal((n_ant, n_samples, 2)) * std
    return np.clip(np.rint(v), -32768, 32767).astype(np.int16)


def gen_delays(rng: np.random.Generator, n_taps: int, max_delay: int) -> np.ndarray:
    """d_0 = 0; the other n_taps-1 drawn without replacement from 1..max_delay, sorted."""
    if n_taps < 1 or n_taps - 1 > max_delay:
        raise ValueError("need 1 <= n_taps <= max_delay + 1")
    rest = rng.choice(np.arange(1, max_delay + 1), size=n_taps - 1, replace=False)
    return np.concatenate([[0], np.sort(rest)]).astype(np.int32)


def pdp_per_tap_decay(n_taps: int, db_per_tap: float = 3.0) -> np.ndarray:
    p = 10.0 ** (-db_per_tap * np.arange(n_taps) / 10.0)
    return p / p.sum()


def pdp_span_decay(delays: np.ndarray, span_db: float = 20.0) -> np.ndarray:
    d = np.asarray(delays, dtype=np.float64)
    dmax = max(float(d.max()), 1.0)
    p = 10.0 ** (-(span_db / 10.0) * d / dmax)
    return p / p.sum()


# ----------------------------------------------------------------------------
# Rayleigh tap processes: sum of sinusoids with Jakes Doppler (Zheng & Xiao 2002)
# ----------------------------------------------------------------------------
def jakes_sos(rng: np.random.Generator, t: np.ndarray, f_d: float, n_proc: int, m: int = 16) -> np.ndarray:
    """n_proc independent unit-power Rayleigh processes sampled at times t (seconds).

    g(t) = m^{-1/2} sum_n [cos(w t cos a_n + phi_n) + j cos(w t sin a_n + psi_n)],
    a_n = (2 pi n - pi + theta) / (4 m), theta, phi_n, psi_n ~ U[-pi, pi).
    Returns complex128 [len(t), n_proc] with E|g|^2 = 1.
    """
    t = np.asarray(t, dtype=np.float64)
    w = 2.0 * np.pi * f_d
    out = np.empty((t.size, n_proc), dtype=np.complex128)
    n = np.arange(1, m + 1, dtype=np.float64)
    for p in range(n_proc):
        theta = rng.uniform(-np.pi, np.pi)
        phi = rng.uniform(-np.pi, np.pi, m)
        psi = rng.uniform(-np.pi, np.pi, m)
        a = (2.0 * np.pi * n - np.pi + theta) / (4.0 * m)
        wt = np.outer(t, w * np.cos(a))
        ws = np.outer(t, w * np.sin(a))
        re = np.cos(wt + phi).sum(axis=1)
        im = np.cos(ws + psi).sum(axis=1)
        out[:, p] = (re + 1j * im) / np.sqrt(m)
    return out


def sos_params(rng: np.random.Generator, f_d: float, pdp: np.ndarray, n_rx: int, n_tx: int, m: int = 16):
    """Random parameters of independent Zheng-Xiao sum-of-sinusoids Rayleigh processes, one per
    (r, t, k) link tap, for synthesis on the device: amplitude sqrt(pdp[k] / n_tx), angular
    frequencies w (cos a_n, sin a_n) with a_n = (2 pi n - pi + theta) / (4 m), phases ~ U[-pi, pi).
    Returns (amplitude float32 [n_rx][n_tx][K], freq float64 [n_rx][n_tx][K][m][2],
    phase float64 [n_rx][n_tx][K][m][2])."""
    k = len(pdp)
    w = 2.0 * np.pi * f_d
    n = np.arange(1, m + 1, dtype=np.float64)
    theta = rng.uniform(-np.pi, np.pi, size=(n_rx, n_tx, k, 1))
    a = (2.0 * np.pi * n - np.pi + theta) / (4.0 * m)
    freq = np.stack([w * np.cos(a), w * np.sin(a)], axis=-1)
    phase = rng.uniform(-np.pi, np.pi, size=(n_rx, n_tx, k, m, 2))
    amp = np.broadcast_to(np.sqrt(np.asarray(pdp, dtype=np.float64) / n_tx), (n_rx, n_tx, k))
    return amp.astype(np.float32), freq, phase


def gen_trace(rng: np.random.Generator, times_s: np.ndarray, f_d: float, pdp: np.ndarray,
              n_rx: int, n_tx: int) -> np.ndarray:
    """Time-varying taps H[a][r][t][k] (complex64) at the given anchor times.

    Every (r, t, k) is an independent Rayleigh process scaled by sqrt(pdp[k] / n_tx),
    so each Rx antenna sees unit total power.
    """
    k = len(pdp)
    g = jakes_sos(rng, times_s, f_d, n_rx * n_tx * k)
    g = g.reshape(len(times_s), n_rx, n_tx, k)
    g *= np.sqrt(np.asarray(pdp, dtype=np.float64) / n_tx)[None, None, None, :]
    return g.astype(np.complex64)


# ----------------------------------------------------------------------------
# Per-UE specification and the workloads
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class UESpec:
    ue_id: int
    n_fft: int
    symbol_len: List[int]
    n_tx: int
    n_rx: int
    delays: np.ndarray          # int32 [K]
    taps: np.ndarray            # complex64 [T][n_rx][n_tx][K]
    step_samples: float = 0.0   # 0: one anchor per symbol
    loop: bool = False
    seed: int = 0
    noise_var: float = 0.0      # sigma^2 per complex sample, 0 = no AWGN
    max_delay: int = 0
    f_d: float = 0.0

    @property
    def n(self) -> int:
        return int(sum(self.symbol_len))

    @property
    def k(self) -> int:
        return int(len(self.delays))

    @property
    def fs(self) -> float:
        return sample_rate(self.n_fft)


def noise_var_for_snr(snr_db: Optional[float]) -> float:
    """sigma^2 = P_x * 10^(-SNR/10) with the nominal input power P_x = 2 * (2^10)^2."""
    if snr_db is None:
        return 0.0
    return P_X_NOMINAL * 10.0 ** (-snr_db / 10.0)


def make_ue(workload: int, ue: int, n_fft: int, n_taps: int, max_delay: int, f_d: float,
            n_slots_trace: int, n_tx: int = 1, n_rx: int = 1, delays: Optional[Sequence[int]] = None,
            pdp: str = "span", snr_db: Optional[float] = None, loop: bool = False,
            seed: Optional[int] = None, step_samples: float = 0.0) -> UESpec:
    L = nr_symbol_lengths(n_fft)
    if delays is None:
        d = gen_delays(rng_for(workload, ue, 0, _S_DELAY), n_taps, max_delay)
    else:
        d = np.asarray(delays, dtype=np.int32)
    p = pdp_per_tap_decay(len(d)) if pdp == "per_tap" else pdp_span_decay(d)
    if step_samples == 0.0:
        n_anchors = 14 * n_slots_trace + 1
        times = anchor_starts(n_anchors, L) / sample_rate(n_fft)
    else:
        n_anchors = int(np.ceil(n_slots_trace * sum(L) / step_samples)) + 2
        times = np.arange(n_anchors) * step_samples / sample_rate(n_fft)
    taps = gen_trace(rng_for(workload, ue, 0, _S_TRACE), times, f_d, p, n_rx, n_tx)
    return UESpec(ue_id=ue, n_fft=n_fft, symbol_len=L, n_tx=n_tx, n_rx=n_rx, delays=d, taps=taps,
                  step_samples=float(step_samples), loop=loop,
                  seed=(SEED_BASE + workload) if seed is None else seed,
                  noise_var=noise_var_for_snr(snr_db), max_delay=max(int(max_delay), int(d.max())),
                  f_d=f_d)


def make_iq(workload: int, spec: UESpec, n_slots: int, first_slot: int = 0) -> np.ndarray:
    """IQ for slots [first_slot, first_slot + n_slots) of one UE: int16 [n_tx][n_slots*N][2]."""
    out = np.empty((spec.n_tx, n_slots * spec.n, 2), dtype=np.int16)
    for t in range(spec.n_tx):
        rng = rng_for(workload, spec.ue_id, t, _S_IQ)
        if first_slot:
            rng.standard_normal((first_slot * spec.n, 2))
        out[t] = gen_iq(rng, 1, n_slots * spec.n)[0]
    return out


def workload_plain_1ue(n_slots: int = 10) -> List[UESpec]:
    """1 UE SISO, 20 MHz (15360 samples/slot), 6 taps {0,3,7,12,20,40}, 3 dB/tap, 10 Hz, no AWGN."""
    return [make_ue(1, 0, 1024, 6, 40, 10.0, n_slots, delays=[0, 3, 7, 12, 20, 40], pdp="per_tap")]


def workload_plain_16ue(n_slots: int = 1000, n_ues: int = 16) -> List[UESpec]:
    """16 UEs SISO, 40 MHz (30720 samples/slot), 24 taps with delays up to 256, 100 Hz, SNR 20 dB."""
    return [make_ue(2, u, 2048, 24, 256, 100.0, n_slots, snr_db=20.0) for u in range(n_ues)]


def workload_batching(n_ues: int = 256, n_slots_trace: int = 20) -> List[UESpec]:
    """UEs of mixed bandwidth {5,20,40,100} MHz in proportion 1:2:4:1, K ~ U{4..48}, d <= 512,
    Doppler ~ U[5, 500] Hz, looping traces."""
    rng = rng_for(3, 1 << 20, 0, 7)
    bws = np.array([5] * 1 + [20] * 2 + [40] * 4 + [100] * 1)
    out = []
    for u in range(n_ues):
        bw = int(bws[u % len(bws)])
        k = int(rng.integers(4, 49))
        f_d = float(rng.uniform(5.0, 500.0))
        out.append(make_ue(3, u, BANDWIDTH_NFFT[bw], k, 512, f_d, n_slots_trace, loop=True,
                           snr_db=20.0))
    return out


def workload_precision(n_ues: int = 64, n_slots_trace: int = 4) -> List[UESpec]:
    """100 MHz, 4x4 MIMO, 96 contiguous taps 0..95 with -20 dB across the span, 100 Hz."""
    return [make_ue(4, u, 4096, 96, 95, 100.0, n_slots_trace, n_tx=4, n_rx=4,
                    delays=np.arange(96), loop=True) for u in range(n_ues)]


def workload_serving(n_ues: int = 512, n_slots_trace: int = 20) -> List[UESpec]:
    """Mixed 20/40/100 MHz, K ~ U{6..48}, half SISO half 2x2, d <= 512, Doppler U[5,500] Hz."""
    rng = rng_for(5, 1 << 20, 0, 7)
    out = []
    for u in range(n_ues):
        bw = int(rng.choice([20, 40, 100]))
        k = int(rng.integers(6, 49))
        mimo = 2 if (u % 2) else 1
        f_d = float(rng.uniform(5.0, 500.0))
        out.append(make_ue(5, u, BANDWIDTH_NFFT[bw], k, 512, f_d, n_slots_trace, n_tx=mimo,
                           n_rx=mimo, loop=True, snr_db=20.0))
    return out
