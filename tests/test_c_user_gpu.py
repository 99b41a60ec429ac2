"""A plain C program (tests/c/tt_chan_c_user.c) drives the library through the C ABI alone.

It streams the 1-UE 20 MHz workload slot by slot (push, run, pull per slot, default ring depth).
Its int16 output must match the FP64 oracle within one LSB, with every mismatch at a rounding tie.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2601_08217_gb300 import inputs
from paper_2601_08217_gb300 import tt_chan as tc
from tests.test_parity_gpu import assert_int16_close

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _write_input(path, spec, x):
    n_slots = x.shape[1] // spec.n
    taps = np.ascontiguousarray(spec.taps.reshape(spec.taps.shape[0], -1)).astype(np.complex64)
    with open(path, "wb") as f:
        f.write(np.array([spec.n, len(spec.symbol_len), len(spec.delays), taps.shape[0], n_slots,
                          int(bool(spec.loop))], dtype="<u4").tobytes())
        f.write(np.asarray(spec.symbol_len, dtype="<u4").tobytes())
        f.write(np.asarray(spec.delays, dtype="<i4").tobytes())
        f.write(taps.view(np.float32).astype("<f4").tobytes())
        f.write(np.ascontiguousarray(x[0]).astype("<i2").tobytes())


def test_c_program_streams_the_1ue_workload(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib_dir = os.path.dirname(tc.LIB_PATH)
    exe = str(tmp_path / "tt_chan_c_user")
    subprocess.run([gcc, "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "c", "tt_chan_c_user.c"), "-o", exe, "-L", lib_dir, "-lttchan",
                    f"-Wl,-rpath,{lib_dir}"], check=True)
    spec = inputs.workload_plain_1ue(10)[0]
    assert spec.n_tx == 1 and spec.n_rx == 1 and spec.noise_var == 0.0 and spec.step_samples == 0.0
    x = inputs.make_iq(1, spec, 10)
    src, dst = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    _write_input(src, spec, x)
    r = subprocess.run([exe, src, dst], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    q = np.fromfile(dst, dtype="<i2").reshape(1, 10 * spec.n, 2)
    y_ref, q_ref = oracle.run_ue(oracle.OracleUE.from_spec(spec), x)
    assert_int16_close(q, y_ref, q_ref)
