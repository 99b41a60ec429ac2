#!/usr/bin/env python3
"""Benchmark of the per-UE time-varying channel convolution on GB300.

Workload (default): 16 UEs SISO at 40 MHz NR (61.44 Msps, 30720 samples per
0.5 ms slot), 1000 slots each, 24-tap Jakes channels (delays <= 256, 100 Hz),
AWGN at 20 dB from Philox4x32-10, int16 IQ in and out, FP32 arithmetic.
One step = every slot of every UE through the whole path (trace anchors,
ingest, interpolated convolution, AWGN, packing, delay-line carry) in the
batched form; the plain one-launch-per-UE-per-slot form is timed beside it.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs its own
16 UEs (weak scaling, no collective on the data path); value = all ranks'
UE-slots / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import queue
import threading
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_UES, N_SLOTS, N_FFT, N_TAPS, D_MAX = 16, 1000, 2048, 24, 256
SLOT_SAMPLES = 30720
# Algorithmic FP32 work per tap-sample (one link, one tap, one output sample): a complex MAC
# (4 FFMA, 8 flop) and the tap's interpolation h = H + tau*dH (2 FP32-pipe operations, counted as
# 2 flop: one add per component).  The roofline fraction is the FP32-pipe instruction rate this
# implies against SMs x 128 lanes x SM clock; the flop and MAC-only fractions are reported beside it.
INSTR_PER_TAP_SAMPLE = 6
FLOP_PER_TAP_SAMPLE = 10
MAC_FLOP_PER_TAP_SAMPLE = 8
FP32_LANES_PER_SM = 128
DISTINCT_IQ_SLOTS = 64        # synthetic IQ slots per UE, cycled through the replay
METRIC = "UE-slots/s and GMAC/s at 1 GB300 vs plain form; p99 slot latency vs 0.5 ms"
# DRAM traffic per full launch from the ncu capture summarised in
# profiles/tt_conv_fp32_kernel_40mhz_16ue.md, valid only for the kernel source it was taken on.
TRAFFIC_BYTES = 3.51e9
TRAFFIC_KERNEL_SHA = "d44ebac8aef3c4f2"
WORKLOAD = ("16 UEs SISO, 40 MHz (30720 samples/slot), 1000 slots each, 24 taps (delays <= 256), "
            "100 Hz Jakes, AWGN 20 dB, int16 IQ, FP32 accumulation")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    out = {"sm_max_mhz": 2070.0, "hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}
    if os.path.exists(p):
        d = json.load(open(p))
        out.update({k: d[k] for k in ("sm_max_mhz", "hbm_gbs", "bf16_tflops", "bf16_tflops_sustained") if k in d})
        out["src"] = "measured"
    return out


def sm_count(device) -> int:
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def alu_roofline(tap_samples_per_launch: float, kernel_ms: float, n_sm: int, clock_mhz: float, clock_src: str):
    """The FP32-pipe roofline of a tiled-kernel launch, every figure derivable from the fields."""
    t = kernel_ms / 1e3
    peak_instr = n_sm * FP32_LANES_PER_SM * clock_mhz * 1e6       # FP32-pipe lane-operations per second
    achieved = tap_samples_per_launch * INSTR_PER_TAP_SAMPLE / t
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_instr / 1e12,
            "unit": "T FP32-pipe instructions/s", "frac": achieved / peak_instr,
            "frac_definition": f"{INSTR_PER_TAP_SAMPLE} algorithmic FP32-pipe instructions per tap-sample "
                               f"(4 FFMA complex MAC + 2 for the interpolation) x tap-samples per launch / "
                               f"kernel time, over SMs x {FP32_LANES_PER_SM} lanes x SM clock",
            "tap_samples_per_launch": tap_samples_per_launch, "kernel_ms": kernel_ms, "sm_count": n_sm,
            "sm_clock_mhz": clock_mhz, "clock_src": clock_src,
            "flop_frac": tap_samples_per_launch * FLOP_PER_TAP_SAMPLE / t / (2 * peak_instr),
            "mac_only_frac": tap_samples_per_launch * MAC_FLOP_PER_TAP_SAMPLE / t / (2 * peak_instr),
            "flop_definition": f"{FLOP_PER_TAP_SAMPLE} flop per tap-sample (8 complex MAC + 2 interpolation) "
                               f"and 8 (MAC only), over SMs x {FP32_LANES_PER_SM} x 2 flop x SM clock"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 20 ms from before the warm-up
    until after the timed region; the summary keeps the samples stamped inside the region."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.rows = []
        self.window = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def region(self, t_begin: float, t_end: float):
        self.window = (t_begin, t_end)

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        import datetime
        for line in out.splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 10:
                continue
            try:
                t = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            self.rows.append((t, f[1:]))

    def summary(self):
        rows = self.rows
        if rows and self.window:
            a, b = self.window
            inside = [r for r in rows if a - 0.02 <= r[0] <= b + 0.02]
            rows = inside or sorted(rows, key=lambda r: abs(r[0] - 0.5 * (a + b)))[:1]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        f = [r[1] for r in rows]
        sm = [float(x[1]) for x in f if x[1].replace(".", "").isdigit()]
        mx = [float(x[2]) for x in f if x[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for x in f for n, v in zip(names, x[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_workload(rank: int, n_slots: int = None, n_ues: int = N_UES, iq_slots: int = DISTINCT_IQ_SLOTS):
    """Rank `rank`'s UEs: the 16-UE workload with AWGN keyed by the global UE ids of its shard."""
    from paper_2601_08217_gb300 import inputs, shard
    specs = inputs.workload_plain_16ue(n_slots=N_SLOTS if n_slots is None else n_slots, n_ues=n_ues)
    for s, uid in zip(specs, shard.shard_ue_ids(n_ues, rank)):
        s.loop = True            # repeated steps keep replaying the trace
        s.ue_id = uid
    iq = [inputs.make_iq(2, s, iq_slots) for s in specs]
    return specs, iq


def whole_job_rate(ms_total: float, steps: int, world: int, ue_slots_per_rank_step: int, device=None):
    """(ms per step of the slowest rank, UE-slots/s of all ranks together): every rank processes
    ue_slots_per_rank_step UE-slots per step, and the job takes as long as its slowest rank."""
    from paper_2601_08217_gb300 import shard
    ms_step = shard.max_over_ranks(ms_total / steps, device=device)
    return ms_step, ue_slots_per_rank_step * world / (ms_step / 1e3)


def cycled_slots(x, n, count, first=0):
    """[count][n_tx][N][2] int16 from the distinct slots of x ([n_tx][D*N][2]), cycled."""
    from paper_2601_08217_gb300 import tt_chan as tc
    sm = tc.slots_major(x, n)
    idx = (np.arange(count) + first) % sm.shape[0]
    return np.ascontiguousarray(sm[idx])


def tap_samples(specs):
    return sum(s.n * len(s.delays) * s.n_tx * s.n_rx for s in specs)


def run_ours(args, rank, world, device):
    import torch
    from paper_2601_08217_gb300 import shard
    from paper_2601_08217_gb300 import tt_chan as tc

    specs, iq = make_workload(rank)
    n = specs[0].n
    eng = tc.Engine(device=device, form="batched", persistent=bool(args.persistent),
                    samples_per_thread=args.spt)
    q = N_SLOTS + 1
    chans = [tc.Chan(eng, s, ring_slots=q) for s in specs]
    stream = torch.cuda.ExternalStream(eng.stream)
    # fill every ring position once (slots 0..1000), then replay in place
    for ch, x in zip(chans, iq):
        ch.push(0, cycled_slots(x, n, N_SLOTS))
    eng.run()
    for ch in chans:
        tc.tt_chan_release_slots(ch.h, 0, N_SLOTS)
    for ch, x in zip(chans, iq):
        ch.push(N_SLOTS, cycled_slots(x, n, 1, N_SLOTS))
    eng.run()
    for ch in chans:
        tc.tt_chan_release_slots(ch.h, N_SLOTS, 1)
    eng.sync()
    next_slot = [N_SLOTS + 1]

    def step(ev=None):
        s0 = next_slot[0]
        for ch in chans:
            tc.tt_chan_commit_slots(ch.h, s0, N_SLOTS)
        if ev is not None:
            ev[0].record(stream)
        eng.run()
        if ev is not None:
            tc.tt_engine_join(eng.h)  # the end event follows every launch lane's batches
            ev[1].record(stream)
        for ch in chans:
            tc.tt_chan_release_slots(ch.h, s0, N_SLOTS)
        next_slot[0] = s0 + N_SLOTS

    clk = ClockSampler(device).start()
    try:
        for _ in range(args.warmup):
            step()
        eng.sync()
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        launches0 = eng.stats()["launches"]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        w0 = time.time()
        t0.record(stream)
        for i in range(args.steps):
            step(kev[i])
        tc.tt_engine_join(eng.h)  # the end event follows every launch lane's batches
        t1.record(stream)
        eng.sync()
        torch.cuda.synchronize()
        clk.region(w0, time.time())
        time.sleep(0.05)
    finally:
        clk.stop()
    if world > 1:
        torch.distributed.barrier()
    launches = eng.stats()["launches"] - launches0
    ms_total = t0.elapsed_time(t1)
    kern_ms = [a.elapsed_time(b) for a, b in kev]

    # ---- e2e through the public API with pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        h_in = [torch.from_numpy(cycled_slots(x, n, N_SLOTS)).pin_memory() for x in iq]
        h_out = [torch.empty((N_SLOTS, 1, n, 2), dtype=torch.int16).pin_memory() for _ in chans]
        e2e_steps = max(1, min(args.steps, 5))
        # slots per push/run/pull round: the copies of one chunk overlap the kernels of the next
        chunk = 125 if N_SLOTS % 125 == 0 else N_SLOTS
        slot_bytes = n * 2 * 2
        hs = [ch.h for ch in chans]

        def e2e_run(n_steps):
            # one continuous stream of n_steps x N_SLOTS slots, as a streaming user drives it: a
            # producer thread pushes chunk after chunk (all UEs in one call, host buffers) and
            # launches it; this thread pulls each launched chunk back to host buffers, so the
            # host-to-device and device-to-host copies overlap each other and the kernels, also
            # across step boundaries.  Every step's input copies and output reads are in the run.
            s0 = next_slot[0]
            total = n_steps * N_SLOTS
            launched = queue.Queue()
            room = threading.Semaphore(4)   # chunks pushed ahead of the pulls (500 of 1001 ring slots)
            err = []

            def producer():
                try:
                    for c0 in range(0, total, chunk):
                        room.acquire()
                        off = (c0 % N_SLOTS) * slot_bytes
                        tc.tt_engine_push_slots(eng.h, hs, [s0 + c0] * len(hs), [chunk] * len(hs),
                                                [hi.data_ptr() + off for hi in h_in])
                        eng.run()
                        launched.put(c0)
                except Exception as ex:  # surfaced below
                    err.append(ex)
                    launched.put(None)

            th = threading.Thread(target=producer, daemon=True)   # never outlives a failed pull
            th.start()
            for _ in range(0, total, chunk):
                c0 = launched.get()
                if c0 is None:
                    break
                off = (c0 % N_SLOTS) * slot_bytes
                tc.tt_engine_pull_slots(eng.h, hs, [s0 + c0] * len(hs), [chunk] * len(hs),
                                        [ho.data_ptr() + off for ho in h_out], -1)
                room.release()
            th.join()
            if err:
                raise err[0]
            next_slot[0] = s0 + total

        e2e_run(1)
        if world > 1:
            torch.distributed.barrier()
        ts = time.perf_counter()
        e2e_run(e2e_steps)
        te = shard.max_over_ranks(time.perf_counter() - ts, device="cuda")
        bytes_in = sum(h.numel() * 2 for h in h_in)
        bytes_out = sum(h.numel() * 2 for h in h_out)
        e2e = {"value": N_UES * N_SLOTS * world * e2e_steps / te, "unit": "UE-slots/s",
               "h2d_bytes_per_step": bytes_in, "d2h_bytes_per_step": bytes_out, "steps": e2e_steps}
    eng.close()

    # ---- plain form on the same GPU, same workload ----
    plain = None
    if not args.no_plain:
        engp = tc.Engine(device=device, form="plain")
        chp = [tc.Chan(engp, s, ring_slots=q) for s in specs]
        for ch, x in zip(chp, iq):
            ch.push(0, cycled_slots(x, n, N_SLOTS))
        sp = torch.cuda.ExternalStream(engp.stream)
        engp.run()
        for ch in chp:
            tc.tt_chan_release_slots(ch.h, 0, N_SLOTS)
        engp.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for ch in chp:
            tc.tt_chan_commit_slots(ch.h, N_SLOTS, N_SLOTS - 1)
        a.record(sp)
        engp.run()
        b.record(sp)
        engp.sync()
        pms = a.elapsed_time(b)
        if world > 1:   # whole-job figure, like the headline: every rank's UEs over the slowest rank's time
            pms = shard.max_over_ranks(pms, device="cuda")
        plain = {"value": N_UES * (N_SLOTS - 1) * world / (pms / 1e3), "unit": "UE-slots/s", "ms_per_step": pms,
                 "launches_per_step": N_UES * (N_SLOTS - 1)}
        engp.close()
    return dict(ms_total=ms_total, kern_ms=kern_ms, launches=launches, clocks=clk.summary(), e2e=e2e,
                plain=plain, specs=specs)


def run_batching(args, device, n_ues=256, steps=400, warmup=20):
    """256 UEs of mixed bandwidth (5/20/40/100 MHz, 1:2:4:1), 4-48 taps, delays <= 512, AWGN 20 dB:
    one slot of every UE per step, one CUDA-graph replay of the persistent kernel per step,
    samples per thread and threads per CTA picked by the engine's autotuner."""
    import torch
    from paper_2601_08217_gb300 import inputs
    from paper_2601_08217_gb300 import tt_chan as tc
    specs = inputs.workload_batching(n_ues=n_ues, n_slots_trace=20)
    eng = tc.Engine(device=device, graphs=True, persistent=True)
    chans, xs = [], []
    for sp in specs:
        hist = -(-int(max(sp.max_delay, int(sp.delays.max()))) // sp.n)
        chans.append(tc.Chan(eng, sp, ring_slots=hist + 9))
        xs.append(tc.slots_major(inputs.make_iq(3, sp, 8), sp.n))
    for ch, x in zip(chans, xs):                     # fill every ring position with synthetic IQ
        ch.push(0, x[np.arange(9) % 8])
    eng.run()
    for ch in chans:
        tc.tt_chan_release_slots(ch.h, 0, 9)
    for ch, x in zip(chans, xs):
        ch.push(9, x[1:2])
    eng.run()
    eng.sync()
    stream = torch.cuda.ExternalStream(eng.stream)

    def timed_replay():
        tc.tt_engine_replay(eng.h, warmup, 1)
        eng.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        tc.tt_engine_replay(eng.h, steps, 1)
        tc.tt_engine_join(eng.h)  # the end event follows every launch lane's batches
        ev1.record(stream)
        eng.sync()
        return ev0.elapsed_time(ev1) / steps

    ms_default = timed_replay()                      # the engine's default geometry, before tuning
    tuned = eng.autotune(reps=3)
    # the tuner's choice per class (samples per thread x threads per CTA = the work item's span)
    choice = {}
    for sp, ch in zip(specs, chans):
        g = ch.geometry()
        bucket = 8
        while bucket < len(sp.delays):
            bucket *= 2
        key = (sp.n, f"{sp.n_tx}x{sp.n_rx}", bucket)
        c = choice.setdefault(key, {"samples_per_slot": sp.n, "antennas": key[1], "taps_up_to": bucket, "ues": 0,
                                    "geometry": set()})
        c["ues"] += 1
        c["geometry"].add(f"S={g['samples_per_thread']} x {g['threads_per_cta']} threads = "
                          f"{g['samples_per_item']} samples per item")
    classes = [dict(v, geometry=sorted(v["geometry"])) for _, v in sorted(choice.items())]
    tc.tt_engine_replay(eng.h, warmup, 1)
    eng.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st0 = eng.stats()
    t_host = time.perf_counter()
    a.record(stream)
    tc.tt_engine_replay(eng.h, steps, 1)
    tc.tt_engine_join(eng.h)  # the end event follows every launch lane's batches
    b.record(stream)
    eng.sync()
    t_host = time.perf_counter() - t_host
    st1 = eng.stats()
    ms = a.elapsed_time(b)
    samples = sum(sp.n for sp in specs)
    tap_s = sum(sp.n * len(sp.delays) * sp.n_tx * sp.n_rx for sp in specs)
    eng.close()
    return {"ues": n_ues, "steps": steps, "ms_per_step": ms / steps, "host_ms_per_step": t_host * 1e3 / steps,
            "ue_slots_per_s": n_ues * steps / (ms / 1e3), "gmac_per_s": tap_s * steps / (ms / 1e3) / 1e9,
            "samples_per_slot_step": samples, "realtime": (ms / steps) <= 0.5,
            # whole-step FP32 work against the ALU peak, launch gaps included
            "roofline": alu_roofline(tap_s, ms / steps, sm_count(device), peaks()["sm_max_mhz"],
                                     "sm_max_mhz of " + peaks()["src"] + " peaks"),
            "graph_launches": st1["graph_launches"] - st0["graph_launches"],
            "graph_builds": st1["graph_builds"], "autotuned_classes": tuned, "tuned_geometry": classes,
            "ms_per_step_before_tuning": ms_default}


def run_serving(args, device, n_ues=512, duration=2.0, warmup=0.2, plain_duration=0.3):
    """512 UEs (20/40/100 MHz, SISO and 2x2, 6-48 taps, delays <= 512), Poisson slot pushes at the
    0.5 ms slot rate with +-50 us jitter, device-resident IQ, 40 GB HBM admission budget,
    continuous batching; the plain one-launch-per-UE-per-slot form served the same way beside it.
    Beside them, the batched form serving 256 UEs of the 40 MHz 24-tap kind (the real-time target
    of at least 256 such UEs with p99 under the 0.5 ms slot)."""
    from paper_2601_08217_gb300 import inputs
    from paper_2601_08217_gb300 import tt_chan as tc
    specs = inputs.workload_serving(n_ues=n_ues, n_slots_trace=10)
    out = {}
    for form, dur in (("batched", duration), ("plain", plain_duration), ("batched_256_40mhz", duration)):
        if form == "batched_256_40mhz":
            specs = inputs.workload_plain_16ue(n_slots=10, n_ues=256)
            form_name, form = form, "batched"
        else:
            form_name = form
        eng = tc.Engine(device=device, form=form, persistent=True, hbm_budget_bytes=40 << 30)
        admitted = refused = 0
        chans = []
        for sp in specs:
            hist = -(-int(max(sp.max_delay, int(sp.delays.max()))) // sp.n)
            try:
                ch = tc.Chan(eng, sp, ring_slots=hist + 12)
            except tc.TTError as ex:
                if ex.status != tc.TT_ERR_NO_MEMORY:
                    raise
                refused += 1
                continue
            admitted += 1
            x = tc.slots_major(inputs.make_iq(5, sp, 4), sp.n)
            ch.push(0, x[np.arange(12) % 4])
            chans.append(ch)
        eng.run()
        for ch in chans:
            tc.tt_chan_release_slots(ch.h, 0, 12)
        eng.sync()
        rep = tc.tt_engine_serve(eng.h, duration_s=dur, warmup_s=warmup, slot_period_us=500.0, jitter_us=50.0,
                                 deadline_us=500.0, seed=11, release_outputs=True)
        st = eng.stats()
        eng.close()
        out[form_name] = {"ues_admitted": admitted, "ues_refused": refused, "hbm_gb": st["hbm_in_use"] / 1e9,
                     "duration_s": dur, "requests": rep["requests"], "completed": rep["completed"],
                     "refused_requests": rep["refused"], "ue_slots_per_s": rep["throughput"],
                     "p50_us": rep["p50_us"], "p99_us": rep["p99_us"], "p999_us": rep["p999_us"],
                     "max_us": rep["max_us"], "deadline_misses": rep["deadline_misses"],
                     "mean_batch": rep["mean_batch"], "batches": rep["batches"],
                     "gpu_us_per_batch": rep["gpu_us_per_batch"], "gpu_busy": rep["gpu_busy"],
                     "stamp_error_us": rep["stamp_error_us"],
                     "latency": "device completion stamp (%globaltimer, calibrated to the host steady clock) "
                                "minus the request's host arrival time"}
    out["p99_under_deadline"] = out["batched"]["p99_us"] < 500.0
    out["p99_under_deadline_256_40mhz"] = out["batched_256_40mhz"]["p99_us"] < 500.0
    out["batched_256_40mhz"]["workload"] = "256 UEs SISO, 40 MHz, 24 taps (delays <= 256), AWGN 20 dB"
    return out


def run_precision(args, device, n_ues=64, n_slots=20, warmup=3, forms=("bf16_tc", "fp16_tc", "fp32")):
    """64 UEs at 100 MHz (61440 samples/slot), 4x4 MIMO, 96 contiguous taps (delays 0..95), 100 Hz:
    block-Toeplitz tensor-core form (BF16 and FP16 operands, FP32 accumulation) beside the FP32
    CUDA-core form on the same inputs; EVM against the FP64 oracle on one UE-slot."""
    import torch
    import oracle
    from paper_2601_08217_gb300 import inputs
    from paper_2601_08217_gb300 import tt_chan as tc
    pk = peaks()
    specs = inputs.workload_precision(n_ues=n_ues, n_slots_trace=4)
    iq = [tc.slots_major(inputs.make_iq(4, sp, 4), sp.n) for sp in specs]
    x0 = inputs.make_iq(4, specs[0], 1)
    y_ref, _ = oracle.run_ue(oracle.OracleUE.from_spec(specs[0]), x0)
    out = {}
    n = specs[0].n
    # tensor-core MMAs issued per slot: per symbol, groups of <= 1536 samples (192 block rows of 8),
    # each group one 128 x N x 16 MMA per K-chunk with N = its block rows rounded up to 16; the
    # 144-wide window per (Tx, part) skips the 16-wide chunks no delay reaches: kc = 9 - (128 - d_max) // 16
    ncols = sum(-(-(-(-min(1536, L - g) // 8)) // 16) * 16 for L in specs[0].symbol_len for g in range(0, L, 1536))
    kc = 9 - (128 - int(np.max(specs[0].delays))) // 16
    exec_flop = n_ues * ncols * (4 * 2 * kc) * 128 * 16 * 2
    useful_flop = n_ues * n * 16 * 96 * 8                        # complex MACs per slot
    for name, prec in (("bf16_tc", tc.TT_BF16_TC), ("fp16_tc", tc.TT_FP16_TC), ("fp32", tc.TT_FP32)):
        if name not in forms:
            continue
        # graph-replaying engines rotate consecutive slots over launch lanes (tensor-core channels too)
        eng = tc.Engine(device=device, persistent=True, graphs=True)
        chans = [tc.Chan(eng, sp, ring_slots=n_slots + 2, precision=prec) for sp in specs]
        for ch, x in zip(chans, iq):
            ch.push(0, x[np.arange(n_slots + 1) % 4])
        eng.run()
        for ch in chans:
            tc.tt_chan_release_slots(ch.h, 0, n_slots + 1)
        eng.sync()
        stream = torch.cuda.ExternalStream(eng.stream)
        tc.tt_engine_replay(eng.h, warmup, 1)
        eng.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tc.tt_engine_replay(eng.h, n_slots, 1)
        tc.tt_engine_join(eng.h)  # the end event follows every launch lane's batches
        b.record(stream)
        eng.sync()
        ms = a.elapsed_time(b) / n_slots
        # EVM of UE 0's first slot against the oracle
        e1 = tc.Engine(device=device)
        c1 = tc.Chan(e1, specs[0], ring_slots=3, cf32=True, precision=prec)
        c1.push(0, x0)
        e1.run()
        y = tc.antenna_major(c1.pull(0, 1))
        e1.close()
        evm = 20 * np.log10(np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref))
        rec = {"ms_per_slot_64ue": ms, "realtime": ms <= 0.5, "ue_slots_per_s": n_ues / (ms / 1e3),
               "useful_tflops": useful_flop / (ms / 1e3) / 1e12, "evm_db_vs_oracle": evm}
        if prec != tc.TT_FP32:
            rec["executed_tflops"] = exec_flop / (ms / 1e3) / 1e12
            pkt = pk.get("bf16_tflops", 1900.0)   # FP16 and BF16 share the dense tensor rate
            rec["roofline"] = {"bound": "tensor", "achieved": rec["executed_tflops"], "peak": pkt,
                               "unit": "TFLOP/s", "frac": rec["executed_tflops"] / pkt,
                               "frac_definition": "MMA flop issued per slot (one 128 x N x 16 MMA per K-chunk "
                                                  "and group, chunks no delay reaches skipped) / time, over "
                                                  "the dense BF16 GEMM peak (" + pk["src"] + ")",
                               "useful_frac": rec["useful_tflops"] / pkt,
                               "executed_flop_per_slot": exec_flop, "useful_flop_per_slot": useful_flop}
        out[name] = rec
        eng.close()
    return out


def run_sparse(args, device, top_n=8, n_slots=200, warmup=3):
    """Sparse convolution (Sec. III-C): the headline workload (16 UEs, 40 MHz, 24 taps, AWGN) with
    only the top_n dominant taps of each symbol and link, beside all 24 taps on the same inputs;
    fidelity as the EVM of the sparse output against the all-taps FP64 oracle on one UE-slot."""
    import torch
    import oracle
    from paper_2601_08217_gb300 import tt_chan as tc
    specs, iq = make_workload(0)
    n = specs[0].n
    out = {}
    for name, tn in (("all_taps", 0), ("top_n", top_n)):
        eng = tc.Engine(device=device, persistent=True, graphs=True)
        # rings of two steps plus the delay line: a step's top-n pre-pass then rewrites only sparse-tap
        # ring positions of steps already finished, so consecutive steps overlap on the launch lanes
        chans = [tc.Chan(eng, sp, ring_slots=2 * n_slots + 2, top_n=tn) for sp in specs]
        for ch, x in zip(chans, iq):
            ch.push(0, cycled_slots(x, n, 2 * n_slots + 1))
        eng.run()
        for ch in chans:
            tc.tt_chan_release_slots(ch.h, 0, 2 * n_slots + 1)
        eng.sync()
        stream = torch.cuda.ExternalStream(eng.stream)
        tc.tt_engine_replay(eng.h, warmup, n_slots)
        eng.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tc.tt_engine_replay(eng.h, 5, n_slots)
        tc.tt_engine_join(eng.h)  # the end event follows every launch lane's batches
        b.record(stream)
        eng.sync()
        ms = a.elapsed_time(b) / 5
        eng.close()
        taps = tn if tn else len(specs[0].delays)
        out[name] = {"taps": taps, "ms_per_step": ms, "ue_slots_per_s": len(specs) * n_slots / (ms / 1e3),
                     "gmac_per_s": len(specs) * n_slots * n * taps / (ms / 1e3) / 1e9}
    # fidelity: UE 0, slot 0, complex64 output of the sparse form against the all-taps oracle
    x0 = cycled_slots(iq[0], n, 1)[0]
    e1 = tc.Engine(device=device)
    c1 = tc.Chan(e1, specs[0], ring_slots=3, cf32=True, top_n=top_n)
    c1.push(0, x0[None])
    e1.run()
    y = tc.antenna_major(c1.pull(0, 1))
    e1.close()
    x0a = tc.antenna_major(x0[None])
    sp0 = specs[0]
    y_all, _ = oracle.run_ue(oracle.OracleUE.from_spec(sp0), x0a)
    y_top, _ = oracle.run_ue(oracle.OracleUE.from_spec(sp0, top_n=top_n), x0a)
    sig = np.linalg.norm(y_all)
    out["top_n"]["evm_db_vs_all_taps"] = float(20 * np.log10(np.linalg.norm(y - y_all) / sig))
    out["top_n"]["nrmse_vs_topn_oracle"] = float(np.linalg.norm(y - y_top) / np.linalg.norm(y_top))
    out["speedup"] = out["all_taps"]["ms_per_step"] / out["top_n"]["ms_per_step"]
    out["workload"] = f"16 UEs x {n_slots} slots, 40 MHz, 24 taps (delays <= 256), AWGN 20 dB; top {top_n} per symbol and link"
    return out


def run_cell(args, device, n_slots=200, warmup=3, steps=5):
    """Uplink aggregation (Sec. III-A): the 16 headline UEs (40 MHz, 24 taps, noise off, complex64
    outputs) summed into one cell with AWGN at 20 dB, int16 out, beside the same 16 UEs without
    the cell; the difference is the aggregation's cost, its traffic 16 x 8 B read + 4 B written
    per cell sample."""
    import torch
    from paper_2601_08217_gb300 import inputs
    from paper_2601_08217_gb300 import tt_chan as tc
    specs, iq = make_workload(0)
    for sp in specs:
        sp.noise_var = 0.0
    n = specs[0].n
    res = {}
    for name, with_cell in (("members_only", False), ("with_cell", True)):
        eng = tc.Engine(device=device, persistent=True, graphs=True)
        cell = tc.Cell(eng, cell_id=0, samples_per_slot=n, ring_slots=n_slots + 1, seed=0x77170002,
                       noise_var=inputs.noise_var_for_snr(20.0)) if with_cell else None
        chans = [tc.Chan(eng, sp, ring_slots=n_slots + 2, cf32=True) for sp in specs]
        if cell:
            for ch in chans:
                cell.attach(ch)
        for ch, x in zip(chans, iq):
            ch.push(0, cycled_slots(x, n, n_slots + 1))
        eng.run()
        if not cell:
            for ch in chans:
                tc.tt_chan_release_slots(ch.h, 0, n_slots + 1)
        eng.sync()
        stream = torch.cuda.ExternalStream(eng.stream)
        tc.tt_engine_replay(eng.h, warmup, n_slots)
        eng.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tc.tt_engine_replay(eng.h, steps, n_slots)
        tc.tt_engine_join(eng.h)  # the end event follows every launch lane's batches
        b.record(stream)
        eng.sync()
        res[name] = a.elapsed_time(b) / steps
        eng.close()
    agg_ms = max(res["with_cell"] - res["members_only"], 1e-6)
    traffic = n_slots * n * (len(specs) * 8 + 4)
    pk = peaks()
    return {"workload": f"{len(specs)} UEs x {n_slots} slots, 40 MHz, 24 taps, summed into one cell (AWGN 20 dB at the cell)",
            "ms_per_step": res["with_cell"], "members_only_ms": res["members_only"],
            "ue_slots_per_s": len(specs) * n_slots / (res["with_cell"] / 1e3),
            "aggregation_ms": agg_ms, "aggregation_bytes": traffic,
            "aggregation_gbs": traffic / (agg_ms / 1e3) / 1e9,
            "aggregation_frac_of_hbm": traffic / (agg_ms / 1e3) / 1e9 / pk.get("hbm_gbs", 6800.0)}


def run_synth(args, device, n_slots=200, warmup=3, steps=5):
    """Tap processes synthesised on the device (sum of 16 sinusoids per tap, Zheng-Xiao
    parameters, 100 Hz) for the 16 headline UEs, beside the same UEs replaying stored traces, one
    entry per OFDM symbol or one per 1 ms (anchors interpolated in FP64 trace time): the time per
    step of each and the HBM each channel's taps take."""
    import torch
    from paper_2601_08217_gb300 import inputs
    from paper_2601_08217_gb300 import tt_chan as tc
    specs, iq = make_workload(0)
    n = specs[0].n
    res = {}
    for mode in ("trace", "trace_1ms", "synthesised"):
        eng = tc.Engine(device=device, persistent=True, graphs=True)
        chans = []
        for u, sp in enumerate(specs):
            # rings of two steps plus the delay line, in every mode: a step's anchor pre-pass then
            # rewrites only positions of steps already finished, so consecutive steps overlap
            ch = tc.Chan(eng, sp, ring_slots=2 * n_slots + 2, load=(mode == "trace"))
            if mode == "trace_1ms":   # the same UE's delays, its taps every 61440 samples (1 ms)
                sp1 = inputs.make_ue(2, sp.ue_id, 2048, N_TAPS, D_MAX, 100.0, n_slots, snr_db=20.0, loop=True,
                                     delays=sp.delays, step_samples=61440.0)
                ch.load_trace(sp1.taps, sp1.delays, sp1.step_samples, True)
            if mode == "synthesised":
                rng = np.random.default_rng([0x77170009, u])
                amp, freq, phase = inputs.sos_params(rng, 100.0, inputs.pdp_span_decay(sp.delays, 20.0), 1, 1)
                tc.tt_chan_load_jakes(ch.h, sp.delays, amp, freq, phase, 61.44e6)
            chans.append(ch)
        for ch, x in zip(chans, iq):
            ch.push(0, cycled_slots(x, n, 2 * n_slots + 1))
        eng.run()
        for ch in chans:
            tc.tt_chan_release_slots(ch.h, 0, 2 * n_slots + 1)
        eng.sync()
        st0 = eng.stats()
        stream = torch.cuda.ExternalStream(eng.stream)
        tc.tt_engine_replay(eng.h, warmup, n_slots)
        eng.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tc.tt_engine_replay(eng.h, steps, n_slots)
        tc.tt_engine_join(eng.h)  # the end event follows every launch lane's batches
        b.record(stream)
        eng.sync()
        res[mode] = {"ms_per_step": a.elapsed_time(b) / steps,
                     "hbm_mb_per_ue": (eng.stats()["hbm_in_use"] / len(specs)) / 1e6}
        eng.close()
    res["workload"] = (f"16 UEs x {n_slots} slots, 40 MHz, 24 taps; stored trace of "
                       f"{specs[0].taps.shape[0]} anchors vs 16-sinusoid synthesis per tap")
    res["synthesis_overhead"] = res["synthesised"]["ms_per_step"] / res["trace"]["ms_per_step"] - 1.0
    res["trace_1ms_overhead"] = res["trace_1ms"]["ms_per_step"] / res["trace"]["ms_per_step"] - 1.0
    return res


def cpu_workload():
    """The CPU baseline's sample: slots 0-7 of every UE of the workload, with the oracle's UEs."""
    import oracle
    from paper_2601_08217_gb300 import inputs
    specs = inputs.workload_plain_16ue(n_slots=8, n_ues=N_UES)
    xs = [inputs.make_iq(2, sp, 8) for sp in specs]
    return specs, [oracle.OracleUE.from_spec(sp) for sp in specs], xs


def cpu_model() -> str:
    """The host CPU's model name as lscpu reports it (best effort)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return f"{line.split(':', 1)[1].strip()}, {os.cpu_count()} logical CPUs"
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return f"{platform.machine()}, {os.cpu_count()} logical CPUs"


def cpu_baseline(budget_s: float = 12.0, work=None, single_core: bool = True):
    """The FP64 oracle as it stands on this host's cores, on a bounded sample of the workload.

    The sample is the first 8 slots of every UE of the workload, repeated in
    passes until about budget_s seconds of CPU work have been timed.
    """
    import oracle
    specs, ues, xs = work if work is not None else cpu_workload()
    per_ue = 8
    t = time.perf_counter()
    passes = 0
    while True:
        for ue, x in zip(ues, xs):
            oracle.run_ue(ue, x, want_y=False)
        passes += 1
        dt = time.perf_counter() - t
        if dt >= budget_s or passes >= 1000:
            break
    n_us = passes * N_UES * per_ue
    cores = oracle.max_threads()
    v = n_us / dt
    cmac = specs[0].n * N_TAPS  # complex MACs per UE-slot
    out = {"value": v, "unit": "UE-slots/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
           "sample": f"slots 0-{per_ue - 1} of all {N_UES} UEs, {passes} pass(es): {n_us} UE-slots, "
                     f"{n_us * cmac / 1e9:.2f} G complex MAC in FP64, {dt:.1f} s",
           "seconds": dt, "gmac_per_s": v * cmac / 1e9,
           "realtime_ues": v / 2000.0}   # a 0.5 ms-slot UE needs 2000 UE-slots/s
    if single_core:
        # one core: a few UEs of the same sample (the thread count is put back afterwards)
        t1 = time.perf_counter()
        n1 = 0
        while True:
            for ue, x in zip(ues[:4], xs[:4]):
                oracle.run_ue(ue, x, want_y=False, nthreads=1)
                n1 += per_ue
            d1 = time.perf_counter() - t1
            if d1 >= min(2.0, budget_s / 4):
                break
        oracle.run_ue(ues[0], xs[0][:, :specs[0].n], want_y=False, nthreads=cores)
        out["single_core"] = {"value": n1 / d1, "unit": "UE-slots/s", "gmac_per_s": n1 / d1 * cmac / 1e9}
    return out


def main():
    global N_SLOTS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--persistent", type=int, default=1, help="1: CTAs claim work items from a device counter")
    ap.add_argument("--spt", type=int, default=16,
                    help="engine samples-per-thread cap for the headline (16: the bulk-throughput setting "
                         "for single-antenna channels; 0: the engine's default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-sparse", action="store_true")
    ap.add_argument("--no-cell", action="store_true")
    ap.add_argument("--no-synth", action="store_true")
    ap.add_argument("--only-precision", default="", help="profiling: run only these precision forms "
                    "(comma list of bf16_tc,fp16_tc,fp32) with --prec-ues UEs and print their record")
    ap.add_argument("--prec-ues", type=int, default=64)
    ap.add_argument("--slots", type=int, default=1000,
                    help="slots per UE per step (smaller for profiling captures)")
    args = ap.parse_args()

    N_SLOTS = args.slots
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # the reference arm is the oracle on the host's cores; rank 0 only
        if rank != 0:
            return
        runs = []
        work = cpu_workload()
        budget = min(4.0, 90.0 / max(args.steps, 1))  # the whole run stays within a couple of minutes
        for _ in range(max(args.warmup, 0)):
            cpu_baseline(budget_s=min(1.0, budget), work=work, single_core=False)
        for _ in range(max(args.steps, 1)):
            runs.append(cpu_baseline(budget_s=budget, work=work, single_core=False))
        v = statistics.median(r["value"] for r in runs)
        ms = statistics.median(r["seconds"] for r in runs) * 1e3
        cb = dict(runs[0])
        cb["value"] = v
        cb.pop("seconds", None)
        print(json.dumps({"metric": METRIC, "value": v, "unit": "UE-slots/s", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "impl": "reference",
                          "config": {"workload": WORKLOAD}, "cpu_baseline": cb,
                          "e2e": {"value": v, "unit": "UE-slots/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    import torch
    if args.only_precision:
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps(run_precision(args, local, n_ues=args.prec_ues, n_slots=4, warmup=1,
                                       forms=tuple(args.only_precision.split(",")))))
        return
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    __graft_entry__.build()

    r = run_ours(args, rank, world, local)
    ms_step, value = whole_job_rate(r["ms_total"], args.steps, world, N_UES * N_SLOTS, device="cuda")
    ts = tap_samples(r["specs"]) * N_SLOTS
    gmac = ts * world / (ms_step / 1e3) / 1e9
    pk = peaks()
    import hashlib
    ksrc = os.path.join(ROOT, "paper_2601_08217_gb300", "csrc", "tt_conv_kernel.cuh")
    ksha = hashlib.sha256(open(ksrc, "rb").read()).hexdigest()[:16]
    traffic = TRAFFIC_BYTES if (ksha == TRAFFIC_KERNEL_SHA and N_SLOTS == 1000) else None
    kms = statistics.mean(r["kern_ms"])
    clk_max = r["clocks"].get("sm_max_mhz")
    roof = alu_roofline(ts, kms, sm_count(local), clk_max or pk["sm_max_mhz"],
                        "clocks.max.sm sampled by nvidia-smi" if clk_max else "sm_max_mhz of " + pk["src"] + " peaks")
    roof.update({"traffic": traffic, "kernel": f"tt_conv_fp32_kernel<{args.spt or 8},1,256,false,128>",
                 "dram_gbs": (traffic / (kms / 1e3) / 1e9) if traffic else None,
                 "dram_frac_of_hbm": (traffic / (kms / 1e3) / 1e9 / pk["hbm_gbs"]) if traffic else None,
                 "hbm_peak_gbs": pk["hbm_gbs"]})
    batching = None
    if rank == 0 and world == 1 and not args.no_batching:
        batching = run_batching(args, local)
    precision = None
    if rank == 0 and world == 1 and not args.no_precision:
        precision = run_precision(args, local)
    sparse = None
    if rank == 0 and world == 1 and not args.no_sparse:
        sparse = run_sparse(args, local)
    cell = None
    if rank == 0 and world == 1 and not args.no_cell:
        cell = run_cell(args, local)
    synth = None
    if rank == 0 and world == 1 and not args.no_synth:
        synth = run_synth(args, local)
    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        serving = run_serving(args, local)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:   # the CPU baseline is an N = 1 figure
        cpu = cpu_baseline()
        cpu.pop("seconds", None)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "UE-slots/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "ues_per_gpu": N_UES, "slots": N_SLOTS,
                   "parallelism": f"{world} GPU(s), UEs sharded across them, no data-path collective",
                   "samples_per_slot": SLOT_SAMPLES, "taps": N_TAPS, "max_delay": D_MAX,
                   "form": "batched, persistent CTAs" + (" (device work counter)" if args.persistent else " (strided)"),
                   "samples_per_thread": args.spt or "engine default (8)",
                   "iq": f"{DISTINCT_IQ_SLOTS} distinct synthetic slots per UE cycled",
                   "l2": "inputs larger than L2 (1.97 GB of IQ read per step per GPU)"},
        "gmac_per_s": gmac, "samples_per_s": N_UES * N_SLOTS * SLOT_SAMPLES * world / (ms_step / 1e3),
        "roofline": roof,
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "e2e": r["e2e"],
        "plain": r["plain"],
        "vs_plain": (value / r["plain"]["value"]) if r["plain"] else None,
        "batching": batching,
        "serving": serving,
        "precision": precision,
        "sparse": sparse,
        "cell": cell,
        "synthesis": synth,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
