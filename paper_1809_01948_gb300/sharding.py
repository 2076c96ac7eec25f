"""Host-side logic of multi-GPU runs (one process per GPU, ``torch.distributed``).

The solve itself does not shard here: every box has one GPU, a single system runs on
one GPU, and several GPUs run independent replicas.  What crosses ranks is
bookkeeping: the batched configuration splits its independent systems between ranks
(no collective on the data path), and timings are combined as the maximum over ranks.
"""
from __future__ import annotations

from typing import List, Sequence

import torch


def shard_systems(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Split independent systems between ``world`` ranks, balancing rows: systems are
    taken largest first and each goes to the rank with the fewest rows so far (ties to
    the lowest rank).  Every system lands on exactly one rank; the split depends only on
    the sizes, so all ranks compute the same one without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]), k))
    load = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += int(sizes[k])
    for part in out:
        part.sort()
    return out


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of ``value`` over all ranks of the default process group (the value
    itself without one).  ``device``: where the reduction tensor lives (CUDA for NCCL,
    CPU for gloo)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
