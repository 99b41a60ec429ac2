"""FP64 CPU oracle for the per-UE channel convolution -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The CUDA library never imports, links or calls it,
and it imports nothing from the CUDA side.

Functions and the passages they follow:

* :func:`run_ue` -- Sec. III-B: ``y_u(t) = x(t) * h_u(t)``, linear convolution per
  receiver with the UE's own time-varying impulse response read from a trace
  (Sec. IV: discrete complex taps on a fixed delay grid per time step), plus
  optional AWGN and int16 packing.  The interpolation, anchor placement,
  noise and rounding readings are stated in ``tt_oracle.c``'s header.
* :func:`run_cell` -- Sec. III-A: uplink aggregation at the gNB, the sum of the
  members' convolved streams plus the cell's own AWGN, then packing.
* :func:`resample_cir` -- Sec. IV: a continuous CIR resampled onto the fixed delay
  grid (band-limited discrete-time equivalent, sum of sincs).
* :func:`sos_taps` -- Sec. IV (3GPP traces with Jakes-based Doppler): sum-of-
  sinusoids tap processes at given times, FP64.
* :func:`philox4x32_10` -- the counter-based generator of Salmon et al. (SC'11).
* :func:`noise` -- one complex AWGN sample from Philox words via Box-Muller.
* :func:`anchor` -- the trace value at one OFDM-symbol anchor.
* :mod:`oracle.brute` -- exact rational brute force for tiny inputs.

Pins: ``tests/test_oracle_pins.py`` and, for the raw Philox words against a library
implementation, ``tests/test_philox_library_pin.py`` (both run with ``-m "not gpu"``).
"""
from .oracle import (OracleUE, anchor, build, lib_path, max_threads, noise, philox4x32_10,  # noqa: F401
                     resample_cir, run_cell, run_ue, sos_taps)
