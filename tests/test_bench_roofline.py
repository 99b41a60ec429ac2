"""CPU checks of the benchmark's roofline arithmetic: the tiled kernel's FP32-pipe fraction is
derivable from the fields of its own JSON object, and equals the figures worked out by hand
for the 16-UE, 40 MHz, 24-tap workload."""
import math

import bench
from paper_2601_08217_gb300 import inputs


def test_tap_samples_of_the_headline_workload():
    specs = inputs.workload_plain_16ue(n_slots=2)      # geometry per slot; the trace length is irrelevant
    assert bench.tap_samples(specs) == 16 * 30720 * 24   # UEs x samples per slot x taps (SISO)


def test_alu_roofline_matches_hand_arithmetic():
    # 16,000 UE-slots x 30,720 samples x 24 taps = 11.80 G tap-samples in a 4.589 ms launch;
    # 6 FP32-pipe operations each = 15.42 T/s against 152 SMs x 128 lanes x 2.07 GHz = 40.27 T/s.
    tap_samples = 16_000 * 30_720 * 24
    r = bench.alu_roofline(tap_samples, 4.589, 152, 2070.0, "hand")
    assert math.isclose(r["peak"], 40.27392, rel_tol=1e-12)
    assert math.isclose(r["achieved"], 15.4236, rel_tol=1e-4)
    assert math.isclose(r["frac"], 0.38297, rel_tol=1e-4)
    assert math.isclose(r["flop_frac"], 0.38297 * 10 / 12, rel_tol=1e-4)   # 10 flop against 2 x 6
    assert math.isclose(r["mac_only_frac"], 0.38297 * 8 / 12, rel_tol=1e-4)
    assert r["bound"] == "alu" and r["sm_count"] == 152


def test_alu_roofline_fraction_recomputes_from_its_fields():
    for n_sm, mhz, ms in ((152, 2070.0, 4.55), (148, 1965.0, 7.0), (1, 1000.0, 1.0)):
        r = bench.alu_roofline(1.0e9, ms, n_sm, mhz, "x")
        peak = r["sm_count"] * bench.FP32_LANES_PER_SM * r["sm_clock_mhz"] * 1e6
        achieved = r["tap_samples_per_launch"] * bench.INSTR_PER_TAP_SAMPLE / (r["kernel_ms"] / 1e3)
        assert math.isclose(r["frac"], achieved / peak, rel_tol=1e-12)
        assert math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-12)
