"""Multi-GPU sharding of the channel path: UEs are independent (each UE's
convolution is isolated, Sec. III-C), so ranks take disjoint UE sets and
exchange nothing on the data path.  Only the benchmark's timing uses a
collective (max over ranks)."""
from __future__ import annotations

from typing import List


def shard_ue_ids(n_per_rank: int, rank: int) -> List[int]:
    """UE ids owned by `rank` when every rank runs n_per_rank UEs (weak scaling)."""
    return list(range(rank * n_per_rank, (rank + 1) * n_per_rank))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (e.g. elapsed time) across the process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
