"""The C-ABI library loads and exports every declared symbol; no compute without a GPU (CPU only)."""
import ctypes as C
import os

import pytest

import __graft_entry__
from paper_2601_08217_gb300 import tt_chan as tc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return tc.load()


def test_every_declared_function_is_exported(lib):
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            names += tc.header_functions(os.path.join(ROOT, "include", h))
    assert len(names) >= 23
    for n in names:
        assert hasattr(lib, n), f"{n} declared but not exported"


def test_the_bounds_checked_build_exports_the_same_symbols(lib):
    chk = C.CDLL(tc.LIB_CHECKED_PATH)
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            for n in tc.header_functions(os.path.join(ROOT, "include", h)):
                assert hasattr(chk, n), f"{n} missing from the checked build"
    assert chk.tt_engine_get_check(None, None) == tc.TT_ERR_INVALID


def test_abi_version_and_error_string(lib):
    assert tc.tt_abi_version() == 4
    assert isinstance(tc.tt_last_error(), str)


def test_null_arguments_are_rejected_without_touching_cuda(lib):
    assert lib.tt_engine_run(None) == tc.TT_ERR_INVALID
    assert lib.tt_chan_destroy(None) == tc.TT_ERR_INVALID
    assert lib.tt_chan_get_geometry(None, None) == tc.TT_ERR_INVALID
    assert lib.tt_engine_create(None, None) == tc.TT_ERR_INVALID
    assert "bad config" in tc.tt_last_error()


def test_no_cpu_fallback_without_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tc.TTError) as ei:
        tc.tt_engine_create(0)
    assert ei.value.status == tc.TT_ERR_CUDA


def _static_chan(**over):
    """A tt_conv_static channel description whose device addresses are never dereferenced: every
    case below fails the host-side checks, which run before the call touches CUDA."""
    c = dict(symbol_len=[64, 64], n_tx=1, n_rx=1, ring_slots=4, d_ring_in=0x10000, d_ring_out=0x20000,
             d_taps=0x30000, delays=[0, 3, 70], n_anchors=5, first_slot=0, n_slots=2)
    c.update(over)
    return c


@pytest.mark.parametrize("over,msg", [
    (dict(d_ring_in=0x10008), "16-byte aligned"),                       # 8-byte offset inside a pool
    (dict(d_ring_in=0x10002), "16-byte aligned"),
    (dict(d_taps=0x30004), "d_taps 8-byte"),
    (dict(d_ring_out=0x20002), "d_ring_out 4-byte"),
    (dict(d_ring_out=0x20004, output_format=tc.TT_OUT_CF32), "d_ring_out 8-byte"),
    (dict(ring_slots=2), "history"),       # 2 slots + 1 history slot (delay 70 of N = 128) need 3
    (dict(ring_slots=5, n_slots=5), "history"),
])
def test_static_entry_rejects_before_touching_the_device(lib, over, msg):
    with pytest.raises(tc.TTError) as ei:
        tc.tt_conv_static([_static_chan(**over)])
    assert ei.value.status == tc.TT_ERR_INVALID and msg in str(ei.value)


def test_static_entry_minimum_ring_passes_the_host_checks(lib):
    """ring_slots = n_slots + history is accepted by the host checks; without a GPU the call then
    stops at the device lookup (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the call would launch on the placeholder addresses")
    with pytest.raises(tc.TTError) as ei:
        tc.tt_conv_static([_static_chan(ring_slots=3)])
    assert ei.value.status == tc.TT_ERR_CUDA
