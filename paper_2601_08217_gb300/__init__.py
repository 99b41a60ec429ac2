"""GB300-native engine for per-UE time-varying multi-tap channel convolution.

The compute path lives in ``csrc/`` (CUDA kernels for sm_103a and the C ABI of
``include/tt_chan.h``), built into ``_build/libttchan.so`` by :mod:`.build`.
:mod:`.tt_chan` is the thin Python binding; :mod:`.inputs` draws seeded
synthetic IQ and channel traces.
"""
__version__ = "0.1.0"
