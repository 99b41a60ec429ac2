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


def test_single_process_needs_no_group():
    assert shard.max_over_ranks(2.5) == 2.5
    assert shard.shard_ue_ids(4, 0) == [0, 1, 2, 3]
