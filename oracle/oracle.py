"""ctypes wrapper around the plain-C FP64 oracle (tt_oracle.c). TEST INFRASTRUCTURE ONLY."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tt_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libttoracle.so")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile tt_oracle.c with gcc (-O2, OpenMP) into oracle/_build/libttoracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _UE(C.Structure):
    _fields_ = [
        ("n", C.c_uint32), ("nsym", C.c_uint32), ("sym_len", C.POINTER(C.c_uint32)),
        ("n_tx", C.c_uint32), ("n_rx", C.c_uint32), ("n_taps", C.c_uint32),
        ("delays", C.POINTER(C.c_int32)), ("taps", C.POINTER(C.c_float)),
        ("n_anchors", C.c_uint32), ("step_samples", C.c_double), ("loop", C.c_int32),
        ("seed", C.c_uint64), ("ue_id", C.c_uint32), ("noise_var", C.c_double),
        ("top_n", C.c_uint32), ("keep", C.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            lib.tto_run.argtypes = [C.POINTER(_UE), C.c_uint64, C.c_uint32, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int]
            lib.tto_run.restype = C.c_int
            lib.tto_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            lib.tto_noise.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_double,
                                      C.c_void_p]
            lib.tto_anchor.argtypes = [C.POINTER(_UE), C.c_uint64, C.c_void_p]
            lib.tto_max_threads.restype = C.c_int
            lib.tto_cell.argtypes = [C.c_uint32, C.c_void_p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint64,
                                     C.c_uint32, C.c_double, C.c_void_p, C.c_void_p]
            lib.tto_cell.restype = C.c_int
            _lib = lib
    return _lib


class OracleUE:
    """Keeps the numpy arrays alive that the C struct points into."""

    def __init__(self, symbol_len: Sequence[int], n_tx: int, n_rx: int, delays, taps,
                 step_samples: float = 0.0, loop: bool = False, seed: int = 0, ue_id: int = 0,
                 noise_var: float = 0.0, top_n: int = 0):
        self.sym_len = np.ascontiguousarray(symbol_len, dtype=np.uint32)
        self.delays = np.ascontiguousarray(delays, dtype=np.int32)
        t = np.asarray(taps)
        if np.iscomplexobj(t):
            t = t.astype(np.complex64)
        self.taps = np.ascontiguousarray(t).view(np.float32).reshape(-1)
        k = len(self.delays)
        n_anchors = self.taps.size // (2 * n_rx * n_tx * k)
        if n_anchors * 2 * n_rx * n_tx * k != self.taps.size:
            raise ValueError("taps size does not match [T][n_rx][n_tx][K]")
        self.s = _UE(n=int(self.sym_len.sum()), nsym=len(self.sym_len),
                     sym_len=self.sym_len.ctypes.data_as(C.POINTER(C.c_uint32)),
                     n_tx=n_tx, n_rx=n_rx, n_taps=k,
                     delays=self.delays.ctypes.data_as(C.POINTER(C.c_int32)),
                     taps=self.taps.ctypes.data_as(C.POINTER(C.c_float)), n_anchors=n_anchors,
                     step_samples=float(step_samples), loop=int(bool(loop)), seed=int(seed),
                     ue_id=int(ue_id), noise_var=float(noise_var), top_n=int(top_n))

    @classmethod
    def from_spec(cls, spec, top_n: int = 0) -> "OracleUE":
        return cls(spec.symbol_len, spec.n_tx, spec.n_rx, spec.delays, spec.taps,
                   spec.step_samples, spec.loop, spec.seed, spec.ue_id, spec.noise_var, top_n)


def run_ue(ue: OracleUE, x: np.ndarray, s_first: int = 0, nthreads: int = 0,
           want_y: bool = True, want_q: bool = True, keep: Optional[np.ndarray] = None):
    """Run slots [s_first, s_first + n_slots) of one UE; x is int16 [n_tx][n_slots*N][2].

    keep: None (the UE's top-n rule), or an explicit tap selection bool [n_slots*nsym + 1][n_rx][n_tx][K]
    that replaces it, anchor s_first*nsym + i at position i.
    Returns (y, q): y complex128 [n_rx][n_slots*N] (or None), q int16 [n_rx][n_slots*N][2] (or None).
    """
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.int16)
    n = ue.s.n
    if x.ndim != 3 or x.shape[0] != ue.s.n_tx or x.shape[2] != 2 or x.shape[1] % n:
        raise ValueError("x must be int16 [n_tx][n_slots*N][2]")
    n_slots = x.shape[1] // n
    y = np.empty((ue.s.n_rx, x.shape[1], 2), dtype=np.float64) if want_y else None
    q = np.empty((ue.s.n_rx, x.shape[1], 2), dtype=np.int16) if want_q else None
    km = None
    if keep is not None:
        km = np.ascontiguousarray(keep, dtype=np.uint8)
        want = (n_slots * ue.s.nsym + 1, ue.s.n_rx, ue.s.n_tx, ue.s.n_taps)
        if km.shape != want:
            raise ValueError(f"keep must be {want}")
    s = _UE.from_buffer_copy(ue.s)
    s.keep = None if km is None else km.ctypes.data
    rc = lib.tto_run(C.byref(s), s_first, n_slots, x.ctypes.data,
                     None if y is None else y.ctypes.data, None if q is None else q.ctypes.data,
                     int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    yc = None if y is None else (y[..., 0] + 1j * y[..., 1])
    return yc, q


def run_cell(members, xs, seed: int, cell_id: int, noise_var: float = 0.0, s_first: int = 0):
    """Uplink aggregation at a cell: the members' outputs (each an OracleUE with its own noise off,
    all with the cell's samples per slot and Rx antenna count) summed in member order, plus the
    cell's AWGN keyed by (seed, cell_id), then packed.  xs[u] is member u's int16 input.
    Returns (y complex128 [n_rx][n_slots*N], q int16 [n_rx][n_slots*N][2])."""
    lib = _load()
    ys = []
    for ue, x in zip(members, xs):
        if ue.s.noise_var != 0.0:
            raise ValueError("cell members carry no noise of their own")
        yc, _ = run_ue(ue, x, s_first=s_first, want_q=False)
        ys.append(np.ascontiguousarray(np.stack([yc.real, yc.imag], axis=-1)))
    n_rx, total = ys[0].shape[0], ys[0].shape[1]
    if any(v.shape != ys[0].shape for v in ys):
        raise ValueError("members differ in Rx antennas or length")
    ptrs = (C.c_void_p * len(ys))(*[v.ctypes.data for v in ys])
    y = np.empty((n_rx, total, 2), dtype=np.float64)
    q = np.empty((n_rx, total, 2), dtype=np.int16)
    rc = lib.tto_cell(len(ys), C.cast(ptrs, C.c_void_p), n_rx, total, s_first * members[0].s.n, seed, cell_id,
                      float(noise_var), y.ctypes.data, q.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return y[..., 0] + 1j * y[..., 1], q


def philox4x32_10(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib.tto_philox4x32_10(c.ctypes.data, k.ctypes.data, o.ctypes.data)
    return o


def noise(seed: int, ue_id: int, rx: int, m: int, noise_var: float) -> complex:
    lib = _load()
    o = np.zeros(2, dtype=np.float64)
    lib.tto_noise(seed, ue_id, rx, m, noise_var, o.ctypes.data)
    return complex(o[0], o[1])


def anchor(ue: OracleUE, a: int) -> np.ndarray:
    """H[a] as complex128 [n_rx][n_tx][K]."""
    lib = _load()
    per = ue.s.n_rx * ue.s.n_tx * ue.s.n_taps
    o = np.zeros(2 * per, dtype=np.float64)
    lib.tto_anchor(C.byref(ue.s), a, o.ctypes.data)
    return (o[0::2] + 1j * o[1::2]).reshape(ue.s.n_rx, ue.s.n_tx, ue.s.n_taps)


def max_threads() -> int:
    return int(_load().tto_max_threads())


def resample_cir(gains: np.ndarray, delays: np.ndarray, n_taps: int) -> np.ndarray:
    """Continuous CIR -> taps on the integer delay grid 0 .. n_taps-1 for each time step
    (Sec. IV, 'Tiny-Twin compatible channel traces': a resampling onto a fixed delay grid; the
    paper does not name the method).  The reading is the band-limited discrete-time equivalent of
    a multipath channel (Tse and Viswanath, Fundamentals of Wireless Communication, Sec. 2.2.3):
        h[t][r][x][k] = sum_p a[t][r][x][p] * sinc(k - tau[t][p]),   sinc(v) = sin(pi v) / (pi v),
    with tau in samples (delay x sampling rate).  FP64; sinc is exactly 1 at v = 0 and exactly 0 at
    the other integers.

    gains: complex [T][n_rx][n_tx][P]; delays: [T][P] samples.  Returns complex128 [T][n_rx][n_tx][n_taps].
    """
    g = np.asarray(gains, dtype=np.complex128)
    tau = np.asarray(delays, dtype=np.float64)
    k = np.arange(n_taps, dtype=np.float64)
    v = k[None, None, :] - tau[:, :, None]                     # [T][P][K]
    whole = v == np.round(v)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(whole, (v == 0).astype(np.float64), np.sin(np.pi * v) / (np.pi * v))
    return np.einsum("trxp,tpk->trxk", g, s)


def sos_taps(amplitude: np.ndarray, freq: np.ndarray, phase: np.ndarray, times_s: np.ndarray) -> np.ndarray:
    """Sum-of-sinusoids tap processes (the Jakes-based Doppler model of Sec. IV's 3GPP traces):
        H[t][r][x][k] = amplitude[r][x][k] * M^(-1/2) * sum_n [cos(freq[..][n][0] t + phase[..][n][0])
                                                          + j cos(freq[..][n][1] t + phase[..][n][1])]
    at the given times (seconds); freq in rad/s.  FP64.  With freq = w (cos a_n, sin a_n) and
    a_n = (2 pi n - pi + theta) / (4 M) this is the model of Zheng and Xiao (IEEE Commun. Lett. 2002).

    amplitude [n_rx][n_tx][K]; freq, phase [n_rx][n_tx][K][M][2].  Returns complex128 [T][n_rx][n_tx][K].
    """
    t = np.asarray(times_s, dtype=np.float64)
    f = np.asarray(freq, dtype=np.float64)
    p = np.asarray(phase, dtype=np.float64)
    m = f.shape[3]
    arg_i = t[:, None, None, None, None] * f[None, ..., 0] + p[None, ..., 0]
    arg_q = t[:, None, None, None, None] * f[None, ..., 1] + p[None, ..., 1]
    s = np.cos(arg_i).sum(axis=-1) + 1j * np.cos(arg_q).sum(axis=-1)
    return np.asarray(amplitude, dtype=np.float64)[None] * s / np.sqrt(m)
