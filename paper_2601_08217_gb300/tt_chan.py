"""Thin ctypes binding of libttchan.so (the C ABI in include/tt_chan.h).

Argument marshalling only: every step of the channel path runs in the CUDA
library.  Functions keep the C names (``tt_engine_create`` ...); ``Engine`` and
``Chan`` are small conveniences over them.  If the library has not been built
the binding raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libttchan.so")
LIB_CHECKED_PATH = os.path.join(HERE, "_build", "libttchan_checked.so")  # loaded when TT_CHECKED=1
HEADER = os.path.join(os.path.dirname(HERE), "include", "tt_chan.h")

TT_OK, TT_ERR_INVALID, TT_ERR_NO_MEMORY, TT_ERR_CUDA = 0, -1, -2, -3
TT_ERR_TRACE, TT_ERR_AGAIN, TT_ERR_TIMEOUT, TT_ERR_STATE, TT_ERR_IO = -4, -5, -6, -7, -8
TT_FORM_BATCHED, TT_FORM_PLAIN = 0, 1
TT_FP32, TT_BF16_TC, TT_FP16_TC = 0, 1, 2
TT_OUT_INT16, TT_OUT_CF32 = 0, 1

STATUS_NAMES = {0: "TT_OK", -1: "TT_ERR_INVALID", -2: "TT_ERR_NO_MEMORY", -3: "TT_ERR_CUDA",
                -4: "TT_ERR_TRACE", -5: "TT_ERR_AGAIN", -6: "TT_ERR_TIMEOUT", -7: "TT_ERR_STATE",
                -8: "TT_ERR_IO"}


class TTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


DEV_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
DEV_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class EngineConfig(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("device", C.c_int32), ("hbm_budget_bytes", C.c_uint64),
                ("form", C.c_uint32), ("max_ues", C.c_uint32), ("samples_per_thread", C.c_uint32),
                ("threads_per_block", C.c_uint32), ("persistent", C.c_uint32), ("graphs", C.c_uint32),
                ("dev_alloc", DEV_ALLOC_FN), ("dev_free", DEV_FREE_FN), ("alloc_ctx", C.c_void_p)]


class TorchAllocator:
    """Allocator hook backed by PyTorch's caching allocator: the engine's device buffers then come
    from (and return to) the same pool as the harness's tensors.  Keep the object alive as long as
    the engine (the C side holds its callbacks).  Counts live allocations for tests."""

    def __init__(self, device: int = 0):
        import torch
        self.device = device
        self.live = {}

        def alloc(nbytes, _ctx):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device)
            except Exception:  # out of memory: the engine reports the failure
                return None
            self.live[p] = int(nbytes)
            return p

        def free(ptr, _ctx):
            self.live.pop(ptr, None)
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = DEV_ALLOC_FN(alloc)
        self.free_fn = DEV_FREE_FN(free)

    @property
    def live_bytes(self) -> int:
        return sum(self.live.values())


class ChanConfig(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("ue_id", C.c_uint32), ("samples_per_slot", C.c_uint32),
                ("symbols_per_slot", C.c_uint32), ("symbol_len", C.POINTER(C.c_uint32)),
                ("n_tx", C.c_uint32), ("n_rx", C.c_uint32), ("max_taps", C.c_uint32),
                ("max_delay", C.c_uint32), ("ring_slots", C.c_uint32), ("seed", C.c_uint64),
                ("noise_var", C.c_float), ("precision", C.c_uint32), ("output_format", C.c_uint32),
                ("top_n", C.c_uint32)]


class CellConfig(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("cell_id", C.c_uint32), ("samples_per_slot", C.c_uint32),
                ("n_rx", C.c_uint32), ("ring_slots", C.c_uint32), ("output_format", C.c_uint32),
                ("seed", C.c_uint64), ("noise_var", C.c_float), ("reserved", C.c_uint32)]


class CirDesc(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("n_steps", C.c_uint32), ("n_paths", C.c_uint32),
                ("n_taps", C.c_uint32), ("gains", C.POINTER(C.c_float)), ("delays", C.POINTER(C.c_double)),
                ("step_samples", C.c_double), ("loop", C.c_int32), ("reserved", C.c_uint32)]


class JakesDesc(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("n_taps", C.c_uint32), ("n_sinusoids", C.c_uint32),
                ("reserved", C.c_uint32), ("delays", C.POINTER(C.c_int32)), ("amplitude", C.POINTER(C.c_float)),
                ("freq", C.POINTER(C.c_double)), ("phase", C.POINTER(C.c_double)), ("sample_rate_hz", C.c_double)]


class TraceDesc(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("taps", C.POINTER(C.c_float)),
                ("delays", C.POINTER(C.c_int32)), ("n_anchors", C.c_uint32), ("n_taps", C.c_uint32),
                ("step_samples", C.c_double), ("loop", C.c_int32)]


class EngineStats(C.Structure):
    _fields_ = [("hbm_in_use", C.c_uint64), ("hbm_budget", C.c_uint64), ("n_chans", C.c_uint32),
                ("pad", C.c_uint32), ("launches", C.c_uint64), ("slots_processed", C.c_uint64),
                ("graph_builds", C.c_uint64), ("graph_launches", C.c_uint64)]


class ServeConfig(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("max_slots_per_ue", C.c_uint32), ("warmup_s", C.c_double),
                ("duration_s", C.c_double), ("slot_period_us", C.c_double), ("jitter_us", C.c_double),
                ("deadline_us", C.c_double), ("seed", C.c_uint64), ("release_outputs", C.c_uint32),
                ("max_inflight_batches", C.c_uint32)]


class ServeReport(C.Structure):
    _fields_ = [("requests", C.c_uint64), ("refused", C.c_uint64), ("completed", C.c_uint64),
                ("batches", C.c_uint64), ("deadline_misses", C.c_uint64), ("mean_batch", C.c_double),
                ("throughput", C.c_double), ("p50_us", C.c_double), ("p99_us", C.c_double),
                ("p999_us", C.c_double), ("max_us", C.c_double), ("mean_us", C.c_double),
                ("stamp_error_us", C.c_double), ("gpu_us_per_batch", C.c_double), ("gpu_busy", C.c_double)]


class ServerConfig(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("max_inflight_batches", C.c_uint32), ("release_outputs", C.c_uint32),
                ("queue_timeout_us", C.c_int32), ("deadline_us", C.c_double), ("warmup_us", C.c_double),
                ("coalesce_us", C.c_double)]


class ServerReport(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("requests", C.c_uint64), ("completed", C.c_uint64),
                ("queued", C.c_uint64), ("refused", C.c_uint64), ("batches", C.c_uint64),
                ("deadline_misses", C.c_uint64), ("mean_batch", C.c_double), ("p50_us", C.c_double),
                ("p99_us", C.c_double), ("p999_us", C.c_double), ("max_us", C.c_double), ("mean_us", C.c_double),
                ("min_us", C.c_double), ("stamp_error_us", C.c_double), ("gpu_us_per_batch", C.c_double),
                ("gpu_busy", C.c_double)]


class StaticChan(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("ue_id", C.c_uint32), ("samples_per_slot", C.c_uint32),
                ("symbols_per_slot", C.c_uint32), ("symbol_len", C.POINTER(C.c_uint32)),
                ("n_tx", C.c_uint32), ("n_rx", C.c_uint32), ("ring_slots", C.c_uint32),
                ("d_ring_in", C.c_void_p), ("d_ring_out", C.c_void_p), ("d_taps", C.c_void_p),
                ("delays", C.POINTER(C.c_int32)), ("n_anchors", C.c_uint32), ("n_taps", C.c_uint32),
                ("step_samples", C.c_double), ("loop", C.c_int32), ("seed", C.c_uint64),
                ("noise_var", C.c_float), ("output_format", C.c_uint32), ("first_slot", C.c_uint64),
                ("n_slots", C.c_uint32)]


class CheckReport(C.Structure):
    _fields_ = [("checked_build", C.c_uint32), ("violations", C.c_uint32), ("first_code", C.c_uint32),
                ("pad", C.c_uint32)]


class ChanGeometry(C.Structure):
    _fields_ = [("tensor_core", C.c_uint32), ("samples_per_thread", C.c_uint32), ("threads_per_cta", C.c_uint32),
                ("samples_per_item", C.c_uint32), ("items_per_slot", C.c_uint32), ("has_trace", C.c_uint32)]


_VP = C.c_void_p
_SIGS = {
    "tt_engine_create": [C.POINTER(EngineConfig), C.POINTER(_VP)],
    "tt_engine_destroy": [_VP],
    "tt_engine_run": [_VP],
    "tt_engine_run_slot": [_VP],
    "tt_engine_sync": [_VP, C.c_int64],
    "tt_engine_stream": [_VP, C.POINTER(_VP)],
    "tt_engine_get_stats": [_VP, C.POINTER(EngineStats)],
    "tt_engine_autotune": [_VP, C.c_int32, C.POINTER(C.c_uint32)],
    "tt_chan_get_geometry": [_VP, C.POINTER(ChanGeometry)],
    "tt_engine_get_check": [_VP, C.POINTER(CheckReport)],
    "tt_engine_join": [_VP],
    "tt_engine_replay": [_VP, C.c_uint32, C.c_uint32],
    "tt_engine_serve": [_VP, C.POINTER(ServeConfig), C.POINTER(ServeReport)],
    "tt_chan_create": [_VP, C.POINTER(ChanConfig), C.POINTER(_VP)],
    "tt_chan_create_queued": [_VP, C.POINTER(ChanConfig), C.c_int64, C.POINTER(_VP)],
    "tt_server_start": [_VP, C.POINTER(ServerConfig)],
    "tt_server_stop": [_VP, C.POINTER(ServerReport)],
    "tt_chan_destroy": [_VP],
    "tt_chan_load_trace": [_VP, C.POINTER(TraceDesc)],
    "tt_chan_push_slot": [_VP, C.c_uint64, _VP],
    "tt_chan_push_slots": [_VP, C.c_uint64, C.c_uint32, _VP],
    "tt_chan_push_slots_dev": [_VP, C.c_uint64, C.c_uint32, _VP, _VP],
    "tt_chan_push_slot_dev": [_VP, C.c_uint64, _VP, _VP],
    "tt_chan_slot_input": [_VP, C.c_uint64, C.POINTER(_VP)],
    "tt_chan_commit_slots": [_VP, C.c_uint64, C.c_uint32],
    "tt_chan_pull_slot": [_VP, C.POINTER(C.c_uint64), _VP, C.c_int64],
    "tt_chan_pull_slots": [_VP, C.c_uint64, C.c_uint32, _VP, C.c_int64],
    "tt_chan_pull_slots_dev": [_VP, C.c_uint64, C.c_uint32, _VP, _VP],
    "tt_chan_pull_slot_dev": [_VP, C.POINTER(C.c_uint64), _VP, _VP],
    "tt_engine_push_slots": [_VP, C.c_uint32, _VP, _VP, _VP, _VP],
    "tt_cell_create": [_VP, _VP, _VP],
    "tt_chan_load_cir": [_VP, _VP],
    "tt_chan_load_jakes": [_VP, _VP],
    "tt_cell_attach": [_VP, _VP],
    "tt_cell_pull_slots": [_VP, C.c_uint64, C.c_uint32, _VP, C.c_int64],
    "tt_cell_destroy": [_VP],
    "tt_engine_pull_slots": [_VP, C.c_uint32, _VP, _VP, _VP, _VP, C.c_int64],
    "tt_chan_slot_output": [_VP, C.c_uint64, C.POINTER(_VP)],
    "tt_chan_release_slots": [_VP, C.c_uint64, C.c_uint32],
    "tt_chan_get_state": [_VP, _VP, C.POINTER(C.c_size_t)],
    "tt_chan_set_state": [_VP, _VP, C.c_size_t],
    "tt_conv_static": [C.POINTER(StaticChan), C.c_uint32, _VP],
}

_lib = None


def header_functions(path: str = HEADER) -> list:
    """Names of every function the public headers declare."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(tt_\w+)\s*\(", txt, flags=re.M)))


def load(path: Optional[str] = None):
    """Load libttchan.so, or with TT_CHECKED=1 in the environment its bounds-checked build (raises if
    it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or (LIB_CHECKED_PATH if os.environ.get("TT_CHECKED") == "1" else LIB_PATH)
    if not os.path.exists(p):
        raise RuntimeError(f"libttchan.so is not built ({p}); run __graft_entry__.build()")
    lib = C.CDLL(p)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int32
    lib.tt_last_error.restype = C.c_char_p
    lib.tt_last_error.argtypes = []
    lib.tt_abi_version.restype = C.c_int32
    _lib = lib
    return lib


def _check(status: int):
    if status != TT_OK:
        raise TTError(status, (_lib.tt_last_error() or b"").decode(errors="replace"))


def _ptr(x) -> int:
    """Address of a numpy array or a torch tensor (host or device); 0 for None."""
    if x is None:
        return 0
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("buffer must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream_ptr(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ---------------------------------------------------------------- C-named calls
def tt_engine_create(device: int = 0, form: int = TT_FORM_BATCHED, hbm_budget_bytes: int = 0,
                     max_ues: int = 0, samples_per_thread: int = 0, persistent: bool = False,
                     graphs: bool = False, threads_per_block: int = 0, allocator=None) -> int:
    """allocator: None (cudaMalloc) or an object with alloc_fn/free_fn ctypes callbacks (TorchAllocator)."""
    lib = load()
    cfg = EngineConfig(C.sizeof(EngineConfig), device, hbm_budget_bytes, form, max_ues,
                       samples_per_thread, threads_per_block, int(bool(persistent)), int(bool(graphs)))
    if allocator is not None:
        cfg.dev_alloc = allocator.alloc_fn
        cfg.dev_free = allocator.free_fn
    h = _VP()
    _check(lib.tt_engine_create(C.byref(cfg), C.byref(h)))
    return h.value


def tt_engine_destroy(e: int):
    _check(load().tt_engine_destroy(e))


def tt_engine_run(e: int):
    _check(load().tt_engine_run(e))


def tt_engine_run_slot(e: int):
    _check(load().tt_engine_run_slot(e))


def tt_engine_sync(e: int, timeout_us: int = -1):
    _check(load().tt_engine_sync(e, timeout_us))


def tt_engine_stream(e: int) -> int:
    s = _VP()
    _check(load().tt_engine_stream(e, C.byref(s)))
    return s.value or 0


def tt_engine_get_stats(e: int) -> dict:
    st = EngineStats()
    _check(load().tt_engine_get_stats(e, C.byref(st)))
    return {f: getattr(st, f) for f, _ in EngineStats._fields_ if f != "pad"}


def tt_engine_autotune(e: int, reps: int = 3) -> int:
    n = C.c_uint32(0)
    _check(load().tt_engine_autotune(e, reps, C.byref(n)))
    return n.value


def tt_engine_join(e: int):
    _check(load().tt_engine_join(e))


def tt_engine_get_check(e: int) -> dict:
    r = CheckReport()
    _check(load().tt_engine_get_check(e, C.byref(r)))
    return {f: getattr(r, f) for f, _ in CheckReport._fields_ if f != "pad"}


def tt_chan_get_geometry(c: int) -> dict:
    g = ChanGeometry()
    _check(load().tt_chan_get_geometry(c, C.byref(g)))
    return {f: getattr(g, f) for f, _ in ChanGeometry._fields_}


def tt_engine_replay(e: int, n_steps: int, slots_per_step: int = 1):
    _check(load().tt_engine_replay(e, n_steps, slots_per_step))


def tt_engine_serve(e: int, duration_s: float, warmup_s: float = 0.0, slot_period_us: float = 500.0,
                    jitter_us: float = 50.0, deadline_us: float = 500.0, seed: int = 0,
                    max_slots_per_ue: int = 0, release_outputs: bool = True, max_inflight_batches: int = 0) -> dict:
    cfg = ServeConfig(C.sizeof(ServeConfig), max_slots_per_ue, warmup_s, duration_s, slot_period_us, jitter_us,
                      deadline_us, seed, int(bool(release_outputs)), max_inflight_batches)
    rep = ServeReport()
    _check(load().tt_engine_serve(e, C.byref(cfg), C.byref(rep)))
    return {f: getattr(rep, f) for f, _ in ServeReport._fields_}


def tt_server_start(e: int, max_inflight_batches: int = 0, release_outputs: bool = False,
                    queue_timeout_us: int = 0, deadline_us: float = 500.0, warmup_us: float = 0.0,
                    coalesce_us: float = 0.0):
    cfg = ServerConfig(C.sizeof(ServerConfig), max_inflight_batches, int(bool(release_outputs)), queue_timeout_us,
                       deadline_us, warmup_us, coalesce_us)
    _check(load().tt_server_start(e, C.byref(cfg)))


def tt_server_stop(e: int) -> dict:
    rep = ServerReport()
    rep.struct_size = C.sizeof(ServerReport)
    _check(load().tt_server_stop(e, C.byref(rep)))
    return {f: getattr(rep, f) for f, _ in ServerReport._fields_ if f != "struct_size"}


def tt_chan_create(e: int, samples_per_slot: int, symbol_len: Sequence[int], n_tx: int = 1, n_rx: int = 1,
                   max_taps: int = 128, max_delay: int = 0, ring_slots: int = 0, seed: int = 0,
                   noise_var: float = 0.0, ue_id: int = 0, precision: int = TT_FP32,
                   output_format: int = TT_OUT_INT16, top_n: int = 0, wait_us: Optional[int] = None) -> int:
    """wait_us: None = plain admission; else tt_chan_create_queued with that timeout (< 0: no limit)."""
    lib = load()
    L = (C.c_uint32 * len(symbol_len))(*[int(v) for v in symbol_len])
    cfg = ChanConfig(C.sizeof(ChanConfig), ue_id, samples_per_slot, len(symbol_len), L, n_tx, n_rx,
                     max_taps, max_delay, ring_slots, seed, noise_var, precision, output_format, top_n)
    h = _VP()
    if wait_us is None:
        _check(lib.tt_chan_create(e, C.byref(cfg), C.byref(h)))
    else:
        _check(lib.tt_chan_create_queued(e, C.byref(cfg), int(wait_us), C.byref(h)))
    return h.value


def tt_chan_destroy(c: int):
    _check(load().tt_chan_destroy(c))


def tt_chan_load_trace(c: int, taps: np.ndarray, delays, step_samples: float = 0.0, loop: bool = False):
    """taps: complex [n_anchors][n_rx][n_tx][K]; delays: int [K]."""
    taps = np.asarray(taps)
    if taps.ndim != 4 or not np.iscomplexobj(taps):
        raise ValueError("taps must be complex [n_anchors][n_rx][n_tx][K]")
    n_anchors = taps.shape[0]
    t = np.ascontiguousarray(taps.astype(np.complex64)).view(np.float32).reshape(-1)
    d = np.ascontiguousarray(delays, dtype=np.int32)
    k = int(d.size)
    desc = TraceDesc(C.sizeof(TraceDesc), t.ctypes.data_as(C.POINTER(C.c_float)),
                     d.ctypes.data_as(C.POINTER(C.c_int32)), n_anchors, k, float(step_samples), int(bool(loop)))
    _check(load().tt_chan_load_trace(c, C.byref(desc)))


def tt_chan_load_cir(c: int, gains: np.ndarray, delays: np.ndarray, n_taps: int, step_samples: float = 0.0,
                     loop: bool = False):
    """gains: complex64 [T][n_rx][n_tx][P]; delays: [T][P] in samples.  The device resamples the CIR
    onto the delay grid 0 .. n_taps-1 and installs it as the channel's trace."""
    g = np.ascontiguousarray(np.asarray(gains, dtype=np.complex64))
    d = np.ascontiguousarray(np.asarray(delays, dtype=np.float64))
    if g.ndim != 4 or d.shape != (g.shape[0], g.shape[3]):
        raise ValueError("gains must be [T][n_rx][n_tx][P] and delays [T][P]")
    desc = CirDesc(C.sizeof(CirDesc), g.shape[0], g.shape[3], int(n_taps),
                   g.ctypes.data_as(C.POINTER(C.c_float)), d.ctypes.data_as(C.POINTER(C.c_double)),
                   float(step_samples), 1 if loop else 0, 0)
    _check(load().tt_chan_load_cir(c, C.byref(desc)))


def tt_chan_load_jakes(c: int, delays, amplitude: np.ndarray, freq: np.ndarray, phase: np.ndarray,
                       sample_rate_hz: float):
    """Sum-of-sinusoids tap processes synthesised on the device: amplitude [n_rx][n_tx][K],
    freq and phase [n_rx][n_tx][K][M][2] (rad/s, rad)."""
    d = np.ascontiguousarray(np.asarray(delays, dtype=np.int32))
    a = np.ascontiguousarray(np.asarray(amplitude, dtype=np.float32))
    f = np.ascontiguousarray(np.asarray(freq, dtype=np.float64))
    p = np.ascontiguousarray(np.asarray(phase, dtype=np.float64))
    if f.shape != p.shape or f.ndim != 5 or f.shape[:3] != a.shape or f.shape[4] != 2 or a.shape[2] != d.size:
        raise ValueError("amplitude [n_rx][n_tx][K], freq/phase [n_rx][n_tx][K][M][2], delays [K]")
    desc = JakesDesc(C.sizeof(JakesDesc), d.size, f.shape[3], 0, d.ctypes.data_as(C.POINTER(C.c_int32)),
                     a.ctypes.data_as(C.POINTER(C.c_float)), f.ctypes.data_as(C.POINTER(C.c_double)),
                     p.ctypes.data_as(C.POINTER(C.c_double)), float(sample_rate_hz))
    _check(load().tt_chan_load_jakes(c, C.byref(desc)))


def tt_chan_push_slot(c: int, slot: int, iq_in):
    _check(load().tt_chan_push_slot(c, slot, _ptr(iq_in)))


def tt_chan_push_slots(c: int, first: int, n: int, iq_in):
    _check(load().tt_chan_push_slots(c, first, n, _ptr(iq_in)))


def tt_chan_push_slots_dev(c: int, first: int, n: int, d_iq_in, stream=None):
    _check(load().tt_chan_push_slots_dev(c, first, n, _ptr(d_iq_in), _stream_ptr(stream)))


def tt_chan_push_slot_dev(c: int, slot: int, d_iq_in, stream=None):
    _check(load().tt_chan_push_slot_dev(c, slot, _ptr(d_iq_in), _stream_ptr(stream)))


def tt_chan_slot_input(c: int, slot: int) -> int:
    p = _VP()
    _check(load().tt_chan_slot_input(c, slot, C.byref(p)))
    return p.value


def tt_chan_commit_slots(c: int, first: int, n: int):
    _check(load().tt_chan_commit_slots(c, first, n))


def tt_chan_pull_slot(c: int, iq_out, timeout_us: int = -1) -> int:
    s = C.c_uint64()
    _check(load().tt_chan_pull_slot(c, C.byref(s), _ptr(iq_out), timeout_us))
    return s.value


def tt_chan_pull_slots(c: int, first: int, n: int, iq_out, timeout_us: int = -1):
    _check(load().tt_chan_pull_slots(c, first, n, _ptr(iq_out), timeout_us))


def _many(chans, first, n, bufs):
    k = len(chans)
    hs = (C.c_void_p * k)(*chans)
    fs = (C.c_uint64 * k)(*first)
    ns = (C.c_uint32 * k)(*n)
    ps = (C.c_void_p * k)(*[_ptr(b) for b in bufs])
    return k, hs, fs, ns, ps


def tt_engine_push_slots(e: int, chans, first, n, iq_in):
    """Push slots of many channels in one call: entry i is (chans[i], first[i], n[i], iq_in[i])."""
    k, hs, fs, ns, ps = _many(chans, first, n, iq_in)
    _check(load().tt_engine_push_slots(e, k, C.cast(hs, C.c_void_p), C.cast(fs, C.c_void_p),
                                       C.cast(ns, C.c_void_p), C.cast(ps, C.c_void_p)))


def tt_engine_pull_slots(e: int, chans, first, n, iq_out, timeout_us: int = -1):
    """Pull slots of many channels in one call: entry i is (chans[i], first[i], n[i], iq_out[i])."""
    k, hs, fs, ns, ps = _many(chans, first, n, iq_out)
    _check(load().tt_engine_pull_slots(e, k, C.cast(hs, C.c_void_p), C.cast(fs, C.c_void_p),
                                       C.cast(ns, C.c_void_p), C.cast(ps, C.c_void_p), timeout_us))


def tt_chan_pull_slots_dev(c: int, first: int, n: int, d_iq_out, stream=None):
    _check(load().tt_chan_pull_slots_dev(c, first, n, _ptr(d_iq_out), _stream_ptr(stream)))


def tt_chan_pull_slot_dev(c: int, d_iq_out, stream=None) -> int:
    s = C.c_uint64()
    _check(load().tt_chan_pull_slot_dev(c, C.byref(s), _ptr(d_iq_out), _stream_ptr(stream)))
    return s.value


def tt_chan_slot_output(c: int, slot: int) -> int:
    p = _VP()
    _check(load().tt_chan_slot_output(c, slot, C.byref(p)))
    return p.value


def tt_chan_release_slots(c: int, first: int, n: int):
    _check(load().tt_chan_release_slots(c, first, n))


def tt_chan_get_state(c: int) -> bytes:
    lib = load()
    n = C.c_size_t(0)
    _check(lib.tt_chan_get_state(c, None, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(lib.tt_chan_get_state(c, buf, C.byref(n)))
    return buf.raw[: n.value]


def tt_chan_set_state(c: int, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(load().tt_chan_set_state(c, buf, len(blob)))


def tt_conv_static(chans, stream=None):
    """chans: list of dicts with the tt_static_chan fields (device buffers as tensors or addresses,
    symbol_len and delays as host sequences).  Runs on `stream` without allocating."""
    arr = (StaticChan * max(len(chans), 1))()
    keep = []
    for i, c in enumerate(chans):
        L = (C.c_uint32 * len(c["symbol_len"]))(*[int(v) for v in c["symbol_len"]])
        d = np.ascontiguousarray(c["delays"], dtype=np.int32)
        keep += [L, d]
        arr[i] = StaticChan(C.sizeof(StaticChan), int(c.get("ue_id", 0)), int(sum(c["symbol_len"])),
                            len(c["symbol_len"]), L, int(c["n_tx"]), int(c["n_rx"]), int(c["ring_slots"]),
                            _ptr(c["d_ring_in"]), _ptr(c["d_ring_out"]), _ptr(c["d_taps"]),
                            d.ctypes.data_as(C.POINTER(C.c_int32)), int(c["n_anchors"]), int(d.size),
                            float(c.get("step_samples", 0.0)), int(bool(c.get("loop", False))),
                            int(c.get("seed", 0)), float(c.get("noise_var", 0.0)),
                            int(c.get("output_format", TT_OUT_INT16)), int(c["first_slot"]),
                            int(c["n_slots"]))
    _check(load().tt_conv_static(arr, len(chans), _stream_ptr(stream)))


def tt_cell_create(e: int, cell_id: int, samples_per_slot: int, n_rx: int = 1, ring_slots: int = 0,
                   seed: int = 0, noise_var: float = 0.0, output_format: int = TT_OUT_INT16) -> int:
    cfg = CellConfig(C.sizeof(CellConfig), cell_id, samples_per_slot, n_rx, ring_slots, output_format, seed,
                     noise_var, 0)
    h = _VP()
    _check(load().tt_cell_create(e, C.byref(cfg), C.byref(h)))
    return h.value


def tt_cell_attach(cell: int, c: int):
    _check(load().tt_cell_attach(cell, c))


def tt_cell_pull_slots(cell: int, first: int, n: int, out, timeout_us: int = -1):
    _check(load().tt_cell_pull_slots(cell, first, n, _ptr(out), timeout_us))


def tt_cell_destroy(cell: int):
    _check(load().tt_cell_destroy(cell))


def tt_last_error() -> str:
    return (load().tt_last_error() or b"").decode(errors="replace")


def tt_abi_version() -> int:
    return int(load().tt_abi_version())


# ---------------------------------------------------------------- conveniences
class Engine:
    def __init__(self, device: int = 0, form: str = "batched", hbm_budget_bytes: int = 0,
                 max_ues: int = 0, samples_per_thread: int = 0, persistent: bool = False, graphs: bool = False,
                 threads_per_block: int = 0, allocator=None):
        """allocator: None (the engine calls cudaMalloc), "torch" (PyTorch's caching allocator), or a
        TorchAllocator-like object with alloc_fn/free_fn callbacks."""
        f = {"batched": TT_FORM_BATCHED, "plain": TT_FORM_PLAIN}[form]
        if allocator == "torch":
            allocator = TorchAllocator(device)
        self.allocator = allocator  # the C side holds its callbacks: keep them alive with the engine
        self.h = tt_engine_create(device, f, hbm_budget_bytes, max_ues, samples_per_thread, persistent, graphs,
                                  threads_per_block, allocator)
        self.chans = []
        self.cells = []

    def run(self):
        tt_engine_run(self.h)

    def sync(self, timeout_us: int = -1):
        tt_engine_sync(self.h, timeout_us)

    @property
    def stream(self) -> int:
        return tt_engine_stream(self.h)

    def stats(self) -> dict:
        return tt_engine_get_stats(self.h)

    def autotune(self, reps: int = 3) -> int:
        return tt_engine_autotune(self.h, reps)

    def check_report(self) -> dict:
        return tt_engine_get_check(self.h)

    def join(self):
        """The engine stream waits (on the device) for every batch launched so far, on any lane."""
        tt_engine_join(self.h)

    def close(self):
        """Destroy the engine.  The C side frees every channel and cell with it, so their handles are
        cleared here first; a later ``destroy()`` on them is then a no-op rather than a dangling call."""
        if self.h:
            for obj in self.chans + self.cells:
                obj.h = None
            self.chans, self.cells = [], []
            tt_engine_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Chan:
    """One UE link.  ``spec`` is an ``inputs.UESpec`` (or anything with its fields)."""

    def __init__(self, engine: Engine, spec, ring_slots: int = 0, load: bool = True, cf32: bool = False,
                 precision: int = TT_FP32, top_n: int = 0, wait_us: Optional[int] = None):
        self.engine = engine
        self.spec = spec
        self.cf32 = cf32
        self.n = int(sum(spec.symbol_len))
        self.h = tt_chan_create(engine.h, self.n, spec.symbol_len, spec.n_tx, spec.n_rx,
                                max(int(len(spec.delays)), 1), int(max(spec.max_delay, max(spec.delays))),
                                ring_slots, int(spec.seed), float(spec.noise_var), int(spec.ue_id),
                                precision=precision, output_format=TT_OUT_CF32 if cf32 else TT_OUT_INT16,
                                top_n=top_n, wait_us=wait_us)
        engine.chans.append(self)
        if load:
            self.load_trace(spec.taps, spec.delays, spec.step_samples, spec.loop)

    def load_trace(self, taps, delays, step_samples=0.0, loop=False):
        tt_chan_load_trace(self.h, np.asarray(taps), delays, step_samples, loop)

    def push(self, first: int, iq: np.ndarray):
        """iq: int16 [n_slots][n_tx][N][2] (or [n_tx][n_slots*N][2], reordered here)."""
        iq = np.asarray(iq, dtype=np.int16)
        if iq.ndim == 3:
            iq = slots_major(iq, self.n)
        tt_chan_push_slots(self.h, first, iq.shape[0], np.ascontiguousarray(iq))

    def pull(self, first: int, n_slots: int, timeout_us: int = -1) -> np.ndarray:
        """int16 [n_slots][n_rx][N][2], or complex64 [n_slots][n_rx][N] for a TT_OUT_CF32 channel."""
        if self.cf32:
            out = np.empty((n_slots, self.spec.n_rx, self.n), dtype=np.complex64)
        else:
            out = np.empty((n_slots, self.spec.n_rx, self.n, 2), dtype=np.int16)
        tt_chan_pull_slots(self.h, first, n_slots, out, timeout_us)
        return out

    def geometry(self) -> dict:
        return tt_chan_get_geometry(self.h)

    def destroy(self):
        if self.h:
            tt_chan_destroy(self.h)
            self.h = None
            if self in self.engine.chans:
                self.engine.chans.remove(self)


def slots_major(x: np.ndarray, n: int) -> np.ndarray:
    """[ant][n_slots*N][2] -> [n_slots][ant][N][2]."""
    a, tot, _ = x.shape
    return np.ascontiguousarray(x.reshape(a, tot // n, n, 2).transpose(1, 0, 2, 3))


def antenna_major(y: np.ndarray) -> np.ndarray:
    """[n_slots][ant][N](...) -> [ant][n_slots*N](...)."""
    s, a, n = y.shape[:3]
    return np.ascontiguousarray(np.moveaxis(y, 1, 0).reshape((a, s * n) + y.shape[3:]))


class Cell:
    """Uplink aggregation cell: the sum of its members' outputs plus the cell's own AWGN."""

    def __init__(self, engine: Engine, cell_id: int, samples_per_slot: int, n_rx: int = 1, ring_slots: int = 0,
                 seed: int = 0, noise_var: float = 0.0, cf32: bool = False):
        self.engine = engine
        self.n, self.n_rx, self.cf32 = int(samples_per_slot), int(n_rx), cf32
        self.h = tt_cell_create(engine.h, cell_id, samples_per_slot, n_rx, ring_slots, seed, noise_var,
                                TT_OUT_CF32 if cf32 else TT_OUT_INT16)
        engine.cells.append(self)

    def attach(self, chan: "Chan"):
        tt_cell_attach(self.h, chan.h)

    def pull(self, first: int, n_slots: int, timeout_us: int = -1) -> np.ndarray:
        """int16 [n_slots][n_rx][N][2], or complex64 [n_slots][n_rx][N] for a TT_OUT_CF32 cell."""
        if self.cf32:
            out = np.empty((n_slots, self.n_rx, self.n), dtype=np.complex64)
        else:
            out = np.empty((n_slots, self.n_rx, self.n, 2), dtype=np.int16)
        tt_cell_pull_slots(self.h, first, n_slots, out, timeout_us)
        return out

    def destroy(self):
        if self.h:
            tt_cell_destroy(self.h)
            self.h = None
            if self in self.engine.cells:
                self.engine.cells.remove(self)
