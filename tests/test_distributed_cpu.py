"""The host-side multi-rank logic on CPU with the gloo backend and two ranks: the split of
independent batched systems between ranks (no collective on the data path) and the
max-over-ranks timing the benchmark reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1809_01948_gb300.sharding import max_over_ranks, shard_systems  # noqa: E402
import testproblems as tp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard_systems(sizes, world)[rank]
        rows = float(sum(sizes[k] for k in mine))
        # every rank sees the same split without exchanging it: gather the lists to check
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out[rank] = dict(mine=mine, all=gathered, max_rows=max_over_ranks(rows), own_rows=rows,
                         max_rank=max_over_ranks(float(rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_batched_systems_and_take_max():
    sizes = [int(s.A.n) for s in tp.problem_batched_banded(nsys=40, n_lo=100, n_hi=5000, band=32).systems]
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, sizes, out), nprocs=2, join=True)
        res = dict(out)
    a, b = res[0], res[1]
    assert a["all"] == b["all"]                               # one split, computed identically
    assert sorted(a["mine"] + b["mine"]) == list(range(40))   # every system exactly once
    assert a["max_rows"] == b["max_rows"] == max(a["own_rows"], b["own_rows"])
    assert a["max_rank"] == b["max_rank"] == 1.0
    # greedy largest-first balance: the heavier rank carries at most one system more than half
    total = sum(sizes)
    assert max(a["own_rows"], b["own_rows"]) <= total / 2 + max(sizes)


def test_shard_systems_single_process_cases():
    assert shard_systems([5, 3, 2], 1) == [[0, 1, 2]]
    assert shard_systems([], 3) == [[], [], []]
    parts = shard_systems([10, 9, 8, 1, 1, 1], 3)
    assert sorted(k for p in parts for k in p) == list(range(6))
    assert [sum([10, 9, 8, 1, 1, 1][k] for k in p) for p in parts] == [10, 10, 10]
    with pytest.raises(ValueError):
        shard_systems([1], 0)
    assert max_over_ranks(3.5) == 3.5   # no process group: the value itself
