"""World-size-2 gloo run of the multi-rank benchmark path on CPU: disjoint UE shards,
max-over-ranks timing, no data-path collective."""
import os
import socket

import torch.multiprocessing as mp

from paper_2601_08217_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ids = shard.shard_ue_ids(16, rank)
    t = shard.max_over_ranks(1.0 + rank * 0.5)
    dist.barrier()
    q.put((rank, ids, t))
    dist.destroy_process_group()


def test_two_ranks_shard_disjointly_and_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ids0, t0), (r1, ids1, t1) = res
    assert set(ids0).isdisjoint(ids1) and sorted(ids0 + ids1) == list(range(32))
    assert t0 == t1 == 1.5


def _bench_worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs, iq = bench.make_workload(rank, n_slots=1, n_ues=3, iq_slots=1)
    # stand-in for the timed region: rank r's 4 steps took 10 + 30 r ms in all
    ms_step, value = bench.whole_job_rate(10.0 + 30.0 * rank, 4, world, 3 * 1000)
    q.put((rank, [s.ue_id for s in specs], [s.seed for s in specs], ms_step, value))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_multi_rank_reporting_on_two_gloo_ranks():
    """bench.py's own multi-rank code on two ranks: each rank's UEs carry the global ids of its shard
    (so their AWGN streams differ), and the whole-job value is all ranks' UE-slots over the slowest
    rank's time per step, the same on every rank."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, ids0, seeds0, ms0, v0), (_, ids1, seeds1, ms1, v1) = res
    assert ids0 == [0, 1, 2] and ids1 == [3, 4, 5]
    assert seeds0 == seeds1                               # one noise key; the UE id separates streams
    assert ms0 == ms1 == 10.0                             # rank 1: 40 ms over 4 steps
    assert v0 == v1 == 2 * 3 * 1000 / 0.010


def test_single_process_needs_no_group():
    assert shard.max_over_ranks(2.5) == 2.5
    assert shard.shard_ue_ids(4, 0) == [0, 1, 2, 3]
