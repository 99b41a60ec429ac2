"""The bounds-checked build (TT_CHECKED) of the tiled and tensor-core kernels: small parity cases
run clean against the oracle, and an out-of-bounds store provoked through a lowered bound (the store
is then skipped, so nothing outside the buffers is touched) is reported with its code while the GPU
and the engine stay usable.

compute-sanitizer is not used here; the bounds-checked library takes its place for both kernels.
The cases run in a child process (tests/checked_run.py) because a process loads one build of the
library.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_is_clean_on_parity_cases_and_reports_a_planted_violation():
    env = dict(os.environ, TT_CHECKED="1")
    env.pop("TT_TEST_CHECK_SHRINK", None)
    r = subprocess.run([sys.executable, "-m", "tests.checked_run"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    rep = json.loads(r.stdout.strip().splitlines()[-1])
    assert rep["cases"] == 66
    assert rep["planted"]["checked_build"] == 1 and rep["planted"]["first_code"] == 11
    assert rep["planted"]["violations"] == rep["groups"] * 2 and rep["after"]["violations"] == 0
    assert rep["tc_planted"]["first_code"] == 11 and rep["tc_planted"]["violations"] > 0
