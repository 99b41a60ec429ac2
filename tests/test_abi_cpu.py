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


def test_abi_version_and_error_string(lib):
    assert tc.tt_abi_version() == 2
    assert isinstance(tc.tt_last_error(), str)


def test_null_arguments_are_rejected_without_touching_cuda(lib):
    assert lib.tt_engine_run(None) == tc.TT_ERR_INVALID
    assert lib.tt_chan_destroy(None) == tc.TT_ERR_INVALID
    assert lib.tt_engine_create(None, None) == tc.TT_ERR_INVALID
    assert "bad config" in tc.tt_last_error()


def test_no_cpu_fallback_without_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tc.TTError) as ei:
        tc.tt_engine_create(0)
    assert ei.value.status == tc.TT_ERR_CUDA
