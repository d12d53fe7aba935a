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


class _SoftmaxRegression(torch.nn.Module):
    """A stand-in with the classifier's training interface (parameters and
    a mean cross-entropy loss) in plain torch, so the data-parallel host
    logic of sgd.fit runs on CPU ranks."""

    def __init__(self, dim, classes):
        super().__init__()
        g = torch.Generator().manual_seed(0)
        self.W = torch.nn.Parameter(0.1 * torch.randn(classes, dim, generator=g, dtype=torch.float64))
        self.b = torch.nn.Parameter(torch.zeros(classes, dtype=torch.float64))

    def loss(self, x, y):
        return torch.nn.functional.cross_entropy(x.double() @ self.W.T + self.b, y.long())


def _data():
    g = torch.Generator().manual_seed(1)
    x = torch.randn(53, 6, generator=g)
    y = torch.randint(0, 4, (53,), generator=g, dtype=torch.int32)
    return x, y


def _fit_worker(rank, world, port, q):
    from paper_1702_08159_gb300.sgd import fit

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, y = _data()
        m = _SoftmaxRegression(6, 4)
        hist = fit(m, x, y, lr=0.5, batch=5, epochs=3, seed=7)  # last batch of 3: one rank gets 1 row
        q.put((rank, m.W.detach().numpy(), m.b.detach().numpy(), hist))
    finally:
        dist.destroy_process_group()


def test_data_parallel_fit_matches_one_process():
    """Two gloo ranks each take half of every mini-batch and sum weighted
    gradients: both end with the parameters, and the epoch losses, of one
    process training on the whole mini-batches."""
    from paper_1702_08159_gb300.sgd import fit

    x, y = _data()
    ref = _SoftmaxRegression(6, 4)
    ref_hist = fit(ref, x, y, lr=0.5, batch=5, epochs=3, seed=7)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_fit_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, W, b, hist in out:
        assert abs(W - ref.W.detach().numpy()).max() < 1e-12
        assert abs(b - ref.b.detach().numpy()).max() < 1e-12
        assert max(abs(h - r) for h, r in zip(hist, ref_hist)) < 1e-12
