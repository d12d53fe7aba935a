"""Host logic of the data-parallel path: shards cover every sample exactly once
and timing/gradient reductions agree across ranks (gloo, world size 2, CPU)."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1702_08159_gb300.dist import allreduce_grads, max_over_ranks, shard_range, sum_over_ranks


@pytest.mark.parametrize("n", [0, 1, 7, 60000, 60001])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_range_partitions(n, world):
    spans = [shard_range(n, r, world) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == n
    for (a, b), (c, _) in zip(spans, spans[1:]):
        assert b == c
    sizes = [b - a for a, b in spans]
    assert max(sizes) - min(sizes) <= 1


def test_shard_range_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 60001
        lo, hi = shard_range(n, rank, world)
        covered = torch.zeros(n, dtype=torch.int32)
        covered[lo:hi] = 1
        dist.all_reduce(covered)
        mx = max_over_ranks(1.5 + rank)
        total = sum_over_ranks(hi - lo)
        p = torch.nn.Parameter(torch.zeros(3))
        p.grad = torch.full((3,), float(rank + 1))
        allreduce_grads([p])
        q.put((rank, int(covered.min()), int(covered.max()), mx, total, p.grad.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, cmin, cmax, mx, total, grad in out:
        assert cmin == 1 and cmax == 1          # every sample on exactly one rank
        assert mx == 2.5                        # max over ranks
        assert total == 60001
        assert grad == [3.0, 3.0, 3.0]          # 1 + 2
