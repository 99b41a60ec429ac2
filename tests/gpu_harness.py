"""Drive the CUDA library through its C ABI for the parity tests (no method arithmetic here)."""
from __future__ import annotations

import numpy as np

from paper_2601_08217_gb300 import tt_chan as tc


def hist_slots(spec) -> int:
    return -(-int(max(spec.max_delay, int(np.max(spec.delays)))) // spec.n)


def run_gpu(specs, xs, n_slots, first_slot=0, cf32=False, form="batched", spt=0, persistent=False,
            stream_mode=False, ring_slots=None, precision=tc.TT_FP32, top_n=0, tpb=0):
    """Run every UE's slots [first_slot, first_slot + n_slots) and return [n_rx][n_slots*N](...) per UE.

    xs[i] is UE i's int16 input [n_tx][n_slots*N][2]; tpb forces the tiled kernel's threads per
    CTA (0: the engine's choice).  Bulk mode pushes all slots,
    runs once and pulls all; stream mode pushes, runs and pulls slot by slot
    through a small ring.
    """
    eng = tc.Engine(form=form, samples_per_thread=spt, persistent=persistent, threads_per_block=tpb)
    try:
        chans = []
        for sp in specs:
            q = ring_slots if ring_slots else (hist_slots(sp) + 3 if stream_mode else n_slots + hist_slots(sp) + 1)
            chans.append(tc.Chan(eng, sp, ring_slots=q, cf32=cf32, precision=precision,
                                 top_n=top_n[len(chans)] if isinstance(top_n, (list, tuple)) else top_n))
        outs = [[] for _ in specs]
        if stream_mode:
            for s in range(n_slots):
                for ch, x in zip(chans, xs):
                    ch.push(first_slot + s, tc.slots_major(x, ch.n)[s:s + 1])
                eng.run()
                for i, ch in enumerate(chans):
                    outs[i].append(ch.pull(first_slot + s, 1))
            res = [tc.antenna_major(np.concatenate(o, axis=0)) for o in outs]
        else:
            for ch, x in zip(chans, xs):
                ch.push(first_slot, x)
            eng.run()
            res = [tc.antenna_major(ch.pull(first_slot, n_slots)) for ch in chans]
        eng.sync()
        return res
    finally:
        eng.close()
