"""Fused logits, softmax cross-entropy and the adjoint kernels against the FP64 oracle.

Bars: logits max abs error <= 1e-4 (a float32 sum of 2 E d products of
features <= 1 with weights ~0.01..0.1); gradients within 1e-4 of the largest
oracle entry (relative); loss within 1e-5.
"""

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import fastfood as ff
from oracle import training as tr

pytestmark = pytest.mark.gpu


def _tables(plan):
    return ff.plan_tables(plan.d, plan.E, plan.kernel, plan.sigma, t=plan.matern_t or 40,
                          seed=plan.seed)


def _rel(got, ref):
    return float(np.abs(got.astype(np.float64) - ref).max() / max(np.abs(ref).max(), 1e-30))


@pytest.mark.parametrize("d,E,C,n", [(8, 2, 10, 5), (64, 2, 3, 9), (1024, 2, 10, 17),
                                     (1024, 3, 16, 8), (1024, 2, 1, 9), (1024, 2, 9, 23),
                                     (1024, 1, 8, 1), (2048, 1, 1, 3), (256, 4, 7, 33),
                                     (1024, 16, 10, 100), (1024, 3, 10, 1300)])
def test_fused_logits(mck, dev, d, E, C, n):
    # At d = 1024 a batch with fewer 8-row tiles than SMs splits the
    # expansions into chunks (n = 100: 13 tiles, uneven chunks of E = 16);
    # n = 1300 has more tiles than SMs, a ragged last tile and blocks that
    # take two tiles.
    plan = mck.Plan(d, E, "rbf", 1.0, 3)
    x = wl.mnist_like(n, min(d, 784), seed=d)
    W, _ = wl.logit_weights(C, 2 * E * d, seed=1, std=0.05)
    b = np.linspace(-1, 1, C).astype(np.float32)
    T = _tables(plan)
    ref = tr.logits(ff.features(x.astype(np.float64), T), W.astype(np.float64), b.astype(np.float64))
    xd = torch.from_numpy(x).to(dev)
    got = mck.fused_logits(plan, xd, torch.from_numpy(W).to(dev), torch.from_numpy(b).to(dev)).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-4
    nob = mck.fused_logits(plan, xd, torch.from_numpy(W).to(dev)).cpu().numpy()
    assert np.abs(nob - (ref - b)).max() <= 1e-4


def test_fused_logits_matches_materialised_path(mck, dev):
    plan = mck.Plan(1024, 4, "rbf", 1.0, 8)
    x = torch.from_numpy(wl.mnist_like(64, 784, seed=8)).to(dev)
    W = torch.from_numpy(wl.logit_weights(10, plan.num_features, seed=2)[0]).to(dev)
    fused = mck.fused_logits(plan, x, W)
    plain = mck.features(plan, x) @ W.T
    assert (fused - plain).abs().max().item() < 1e-5


def test_softmax_xent(mck, dev):
    g = np.random.default_rng(0)
    l = (g.standard_normal((37, 10)) * 4).astype(np.float32)
    y = wl.labels(37, 10, seed=3)
    loss, dl = mck.softmax_xent(torch.from_numpy(l).to(dev), torch.from_numpy(y).to(dev))
    rl, rdl = tr.softmax_xent(l.astype(np.float64), y)
    assert abs(loss.item() - rl) < 1e-5
    assert np.abs(dl.cpu().numpy() - rdl).max() < 1e-6


def test_softmax_xent_bad_label_row_is_zero(mck, dev):
    l = torch.randn(4, 3, device=dev)
    y = torch.tensor([0, 5, -1, 2], dtype=torch.int32, device=dev)
    loss, dl = mck.softmax_xent(l, y)
    assert torch.all(dl[1] == 0) and torch.all(dl[2] == 0)
    rl, _ = tr.softmax_xent(l[[0, 3]].double().cpu().numpy(), np.array([0, 2]))
    assert abs(loss.item() - rl * 2 / 4) < 1e-5


@pytest.mark.parametrize("d,E,n", [(32, 2, 5), (64, 2, 19), (256, 3, 8), (1024, 2, 9)])
def test_features_backward(mck, dev, d, E, n):
    plan = mck.Plan(d, E, "rbf", 1.0, 21)
    in_dim = min(d, 784) - 1
    x = wl.mnist_like(n, in_dim, seed=d)
    dphi = wl.gaussian(n, 2 * E * d, seed=d + 1)
    T = _tables(plan)
    rdx, rdc, rdg = tr.features_backward(x.astype(np.float64), T, dphi.astype(np.float64))
    dx, dc, dg = mck.features_backward(plan, torch.from_numpy(x).to(dev), torch.from_numpy(dphi).to(dev))
    assert _rel(dx.cpu().numpy(), rdx) < 1e-4
    assert _rel(dc.cpu().numpy(), rdc) < 1e-4
    assert _rel(dg.cpu().numpy(), rdg) < 1e-4


@pytest.mark.parametrize("d,E,C,n", [(64, 2, 3, 6), (1024, 2, 10, 11), (64, 2, 3, 1100),
                                     (32, 3, 16, 300)])
def test_fused_logits_backward(mck, dev, d, E, C, n):
    # n = 1100 at d = 64 splits dW's rows over a cluster of 8 blocks (ragged
    # ranges); d = 32 reduces dCs/dG over 8 float4 columns per block.
    plan = mck.Plan(d, E, "rbf", 1.0, 23)
    x = wl.mnist_like(n, min(d, 784), seed=5)
    W, b = wl.logit_weights(C, 2 * E * d, seed=6, std=0.05)
    y = wl.labels(n, C, seed=7)
    T = _tables(plan)
    o = tr.train_grads(x.astype(np.float64), T, W.astype(np.float64), b.astype(np.float64), y)
    xd, Wd = torch.from_numpy(x).to(dev), torch.from_numpy(W).to(dev)
    dl = torch.from_numpy(o["dlogits"].astype(np.float32)).to(dev)
    g = mck.fused_logits_backward(plan, xd, Wd, dl, need_dx=True)
    for k in ("dx", "dCs", "dG", "dW", "db"):
        assert _rel(g[k].cpu().numpy(), o[k]) < 1e-4, k


def test_fused_logits_backward_partial_requests(mck, dev):
    """db alone (no features recomputed for dW), and dW without db."""
    plan = mck.Plan(128, 3, "rbf", 1.0, 29)
    n, C = 300, 5
    x = wl.mnist_like(n, 100, seed=11)
    W, b = wl.logit_weights(C, 2 * 3 * 128, seed=12, std=0.05)
    y = wl.labels(n, C, seed=13)
    o = tr.train_grads(x.astype(np.float64), _tables(plan), W.astype(np.float64),
                       b.astype(np.float64), y)
    xd, Wd = torch.from_numpy(x).to(dev), torch.from_numpy(W).to(dev)
    dl = torch.from_numpy(o["dlogits"].astype(np.float32)).to(dev)
    g = mck.fused_logits_backward(plan, xd, Wd, dl, need_dCs=False, need_dG=False, need_dW=False)
    assert g["dW"] is None and _rel(g["db"].cpu().numpy(), o["db"]) < 1e-5
    g = mck.fused_logits_backward(plan, xd, Wd, dl, need_db=False)
    assert g["db"] is None and _rel(g["dW"].cpu().numpy(), o["dW"]) < 1e-4


def test_training_step_config3_shape(mck, dev):
    # N=512, d=1024 (784 padded), E=16, 10 classes, learnable C and G, uniform labels.
    from paper_1702_08159_gb300.autograd import McKernelClassifier

    N, d, E, C = 512, 1024, 16, 10
    plan = mck.Plan(d, E, "rbf", 1.0, 42)
    x = wl.mnist_like(N, 784, seed=42)
    y = wl.labels(N, C, seed=42)
    W, b = wl.logit_weights(C, 2 * E * d, seed=42)
    model = McKernelClassifier(plan, C, torch.from_numpy(W), torch.from_numpy(b))
    loss = model.loss(torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev))
    loss.backward()
    T = _tables(plan)
    o = tr.train_grads(x.astype(np.float64), T, W.astype(np.float64), b.astype(np.float64), y)
    assert abs(loss.item() - o["loss"]) < 1e-5
    assert _rel(model.W.grad.cpu().numpy(), o["dW"]) < 1e-4
    assert _rel(model.b.grad.cpu().numpy(), o["db"]) < 1e-4
    assert _rel(model.Cs.grad.cpu().numpy(), o["dCs"]) < 1e-4
    assert _rel(model.G.grad.cpu().numpy(), o["dG"]) < 1e-4


def test_autograd_features_matches_fused(mck, dev):
    from paper_1702_08159_gb300.autograd import FastfoodFeatures, FastfoodLogits

    plan = mck.Plan(256, 2, "rbf", 1.0, 4)
    t = plan.tables()
    x = torch.from_numpy(wl.mnist_like(7, 200, seed=9)).to(dev).requires_grad_(True)
    Cs = torch.from_numpy(t["Cs"]).to(dev).requires_grad_(True)
    G = torch.from_numpy(t["G"]).to(dev).requires_grad_(True)
    W = torch.from_numpy(wl.logit_weights(5, plan.num_features, seed=3)[0]).to(dev).requires_grad_(True)
    b = torch.zeros(5, device=dev, requires_grad=True)
    (FastfoodFeatures.apply(plan, x, Cs, G) @ W.T + b).square().sum().backward()
    g1 = [p.grad.clone() for p in (x, Cs, G, W, b)]
    for p in (x, Cs, G, W, b):
        p.grad = None
    FastfoodLogits.apply(plan, x, Cs, G, W, b).square().sum().backward()
    for a, c in zip(g1, (x.grad, Cs.grad, G.grad, W.grad, b.grad)):
        assert (a - c).abs().max().item() <= 1e-4 * max(a.abs().max().item(), 1e-12)


def test_backward_deterministic(mck, dev):
    plan = mck.Plan(1024, 4, "rbf", 1.0, 42)
    x = torch.from_numpy(wl.mnist_like(200, 784, seed=1)).to(dev)
    dphi = torch.from_numpy(wl.gaussian(200, plan.num_features, seed=2)).to(dev)
    a = mck.features_backward(plan, x, dphi)
    b = mck.features_backward(plan, x, dphi)
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_empty_batch_gradients_are_zero(mck, dev):
    plan = mck.Plan(256, 2, "rbf", 1.0, 4)
    x = torch.empty((0, 200), device=dev)
    dx, dc, dg = mck.features_backward(plan, x, torch.empty((0, plan.num_features), device=dev))
    assert dx.shape == (0, 200) and torch.all(dc == 0) and torch.all(dg == 0)
    W = torch.ones((3, plan.num_features), device=dev)
    g = mck.fused_logits_backward(plan, x, W, torch.empty((0, 3), device=dev))
    assert torch.all(g["dW"] == 0) and torch.all(g["db"] == 0) and torch.all(g["dG"] == 0)
    assert mck.fused_logits(plan, x, W).shape == (0, 3)
