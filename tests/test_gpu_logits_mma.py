"""Fused logits with the tensor-core split-precision contraction
(mck_fused_logits_ex, MCK_FP16_SPLIT) against the FP64 oracle.

Error model: every feature phi (|phi| <= 1) and every weight (class c scaled
by an exact power of two so that max |W_c| lies in [2^14, 2^15)) is written
as hi + lo in fp16, and hi.hi + hi.lo + lo.hi go into an FP32 accumulator.
The dropped lo.lo term and the rounding of lo are each below 2^-22 of the
product (fp16 keeps 11 significant bits, so |x - hi| <= 2^-11 |x| and
|x - hi - lo| <= 2^-22 |x|); over K = 2Ed products of random sign the logit
error grows like sqrt(K) 2^-22 rms|phi W|, about 1e-6 at the 60000 x E = 16
MNIST-shaped workload with W ~ N(0, 0.05) (a bf16 split would leave about
2.5e-5 rms there and miss the bar at the maximum over 600000 logits). The
FP32 accumulation adds rounding of the running sums, ~2^-24 |sum| per add
over K / 128 adds per warp (each two 16-feature steps' products go into
a fresh tensor-core accumulator first: the tensor core's own accumulation
truncates relative to the running value, and accumulating every step into one
accumulator measured 1.6e-5 at E = 2 and 1.7e-4 at E = 16): a few 1e-6, below
the FP32 FMA path's own error (~1e-5 at E = 16), so the two paths differ by up
to a few 1e-5 there.
The tests hold the FP32 fused path's bar, max abs error <= 1e-4 against the
oracle, require the two paths to agree within it, and bound the contraction
alone (against a float64 product of the FP32 features) at E = 2, where both
error sources are a few 1e-6, by CONTRACTION_BOUND.
"""

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import fastfood as ff
from oracle import training as tr

pytestmark = pytest.mark.gpu

BAR = 1e-4                # the fused-logits bar against the FP64 oracle
CONTRACTION_BOUND = 1e-5  # E = 2: the contraction alone, ~3x the error model


def _tables(plan):
    return ff.plan_tables(plan.d, plan.E, plan.kernel, plan.sigma, t=plan.matern_t or 40,
                          seed=plan.seed)


def _oracle(plan, x, W, b):
    return tr.logits(ff.features(x.astype(np.float64), _tables(plan)), W.astype(np.float64),
                     b.astype(np.float64))


@pytest.mark.parametrize("E,C,n", [(2, 10, 17), (3, 16, 8), (2, 1, 9), (2, 9, 23), (1, 8, 1),
                                   (16, 10, 100), (3, 10, 1300), (2, 10, 32), (2, 10, 33),
                                   (3, 10, 3000), (4, 5, 8001)])
def test_matches_oracle(mck, dev, E, C, n):
    # n from 1 to 1300: fewer 16-row tiles than resident blocks, so the
    # expansions are split into chunks with partial logits; 32 and 33: whole
    # tiles, and a one-row ragged tile; 3000 and 8001: hundreds of tiles, the
    # latter more than the resident blocks, so that blocks take two tiles;
    # ragged last tiles throughout. C = 1, 5, 8: one 8-class block of W; 9,
    # 10, 16: two.
    plan = mck.Plan(1024, E, "rbf", 3.0, 5 + E)
    x = wl.mnist_like(n, 784, seed=n)
    W, _ = wl.logit_weights(C, plan.num_features, seed=C, std=0.05)
    b = np.linspace(-1, 1, C).astype(np.float32)
    xd = torch.from_numpy(x).to(dev)
    Wd = torch.from_numpy(W).to(dev)
    got = mck.fused_logits(plan, xd, Wd, torch.from_numpy(b).to(dev), prec="fp16_split")
    ref = _oracle(plan, x, W, b)
    assert float(np.abs(got.cpu().numpy() - ref).max()) <= BAR
    fp32 = mck.fused_logits(plan, xd, Wd, torch.from_numpy(b).to(dev))
    assert (got - fp32).abs().max().item() <= BAR
    nob = mck.fused_logits(plan, xd, Wd, prec="fp16_split").cpu().numpy()
    assert float(np.abs(nob - (ref - b)).max()) <= BAR
    plan.close()


def test_full_size_sampled(mck, dev):
    """The MNIST-shaped headline batch: 60000 rows, E = 16, 10 classes."""
    N = 60000
    x = wl.mnist_like(N, 784, seed=42)
    plan = mck.Plan(1024, 16, "rbf", 3.0, 42)
    W, b = wl.logit_weights(10, plan.num_features, seed=42)
    xd = torch.from_numpy(x).to(dev)
    Wd, bd = torch.from_numpy(W).to(dev), torch.from_numpy(b).to(dev)
    got = mck.fused_logits(plan, xd, Wd, bd, prec="fp16_split")
    fp32 = mck.fused_logits(plan, xd, Wd, bd)
    assert torch.isfinite(got).all()
    rows = np.unique(np.concatenate([[0, 1, 15, 16, 17, 31, 32, 33, N // 2, N - 2, N - 1],
                                     np.random.default_rng(3).integers(0, N, 25)]))
    ref = _oracle(plan, x[rows], W, b)
    assert float(np.abs(got.cpu().numpy()[rows] - ref).max()) <= BAR
    assert (got - fp32).abs().max().item() <= BAR
    plan.close()


def test_contraction_error(mck, dev):
    """The split contraction alone: against float64 W phi of the features the
    FP32 feature kernel writes for the same rows (the producers run the same
    FP32 sequence)."""
    plan = mck.Plan(1024, 2, "rbf", 3.0, 8)
    x = torch.from_numpy(wl.mnist_like(500, 784, seed=8)).to(dev)
    W, _ = wl.logit_weights(10, plan.num_features, seed=8, std=0.05)
    got = mck.fused_logits(plan, x, torch.from_numpy(W).to(dev), prec="fp16_split")
    phi = mck.features(plan, x).cpu().numpy().astype(np.float64)
    ref = phi @ W.astype(np.float64).T
    assert float(np.abs(got.cpu().numpy() - ref).max()) <= CONTRACTION_BOUND


@pytest.mark.parametrize("wscale", [1e4, 1e-4])
def test_weight_scale_invariance(mck, dev, wscale):
    """The per-class power-of-two scaling keeps the relative error of the
    contraction whatever the weights' magnitude (fp16's range alone would
    overflow at 1e4 x and lose the lo halves at 1e-4 x)."""
    plan = mck.Plan(1024, 2, "rbf", 3.0, 9)
    x = wl.mnist_like(50, 784, seed=9)
    W, _ = wl.logit_weights(10, plan.num_features, seed=9, std=0.05)
    W = (W * wscale).astype(np.float32)
    W[3] *= 1e-3  # classes of very different magnitude in one call
    got = mck.fused_logits(plan, torch.from_numpy(x).to(dev), torch.from_numpy(W).to(dev),
                           prec="fp16_split").cpu().numpy()
    ref = _oracle(plan, x, W, np.zeros(10, np.float32))
    scale = np.abs(ref).max(axis=0, keepdims=True)
    assert float((np.abs(got - ref) / scale).max()) <= 1e-5


def test_zero_class_and_learned_tables(mck, dev):
    """A class of zero weights gives exactly its bias; caller-supplied Cs and G
    (learned tables) reach the producers."""
    plan = mck.Plan(1024, 3, "rbf", 3.0, 10)
    x = wl.mnist_like(40, 784, seed=10)
    W, _ = wl.logit_weights(10, plan.num_features, seed=10, std=0.05)
    W[4] = 0.0
    b = np.arange(10, dtype=np.float32)
    T = _tables(plan)
    g = np.random.default_rng(10)
    Cs = (T["Cs"] * (1 + 0.1 * g.standard_normal(T["Cs"].shape))).astype(np.float32)
    G = (T["G"] * (1 + 0.1 * g.standard_normal(T["G"].shape))).astype(np.float32)
    got = mck.fused_logits(plan, torch.from_numpy(x).to(dev), torch.from_numpy(W).to(dev),
                           torch.from_numpy(b).to(dev), Cs=torch.from_numpy(Cs).to(dev),
                           G=torch.from_numpy(G).to(dev), prec="fp16_split").cpu().numpy()
    T2 = dict(T, Cs=Cs.astype(np.float64), G=G.astype(np.float64))
    ref = tr.logits(ff.features(x.astype(np.float64), T2), W.astype(np.float64),
                    b.astype(np.float64))
    assert float(np.abs(got - ref).max()) <= BAR
    assert np.all(got[:, 4] == b[4])


def test_strided_unaligned_rows(mck, dev):
    """x as a strided view whose rows are 781 floats long (not a multiple of 4:
    the producers' scalar loads) at a stride of 800, over three 16-row tiles,
    the last ragged."""
    plan = mck.Plan(1024, 2, "rbf", 3.0, 13)
    n, in_dim, ld = 37, 781, 800
    base = torch.from_numpy(wl.mnist_like(n, ld, seed=13)).to(dev)
    x = base[:, :in_dim]
    W, _ = wl.logit_weights(10, plan.num_features, seed=13, std=0.05)
    got = mck.fused_logits(plan, x, torch.from_numpy(W).to(dev), prec="fp16_split")
    ref = _oracle(plan, x.cpu().numpy(), W, np.zeros(10, np.float32))
    assert float(np.abs(got.cpu().numpy() - ref).max()) <= BAR


def test_deterministic(mck, dev):
    plan = mck.Plan(1024, 4, "rbf", 3.0, 11)
    x = torch.from_numpy(wl.mnist_like(3000, 784, seed=11)).to(dev)
    W = torch.from_numpy(wl.logit_weights(10, plan.num_features, seed=11)[0]).to(dev)
    a = mck.fused_logits(plan, x, W, prec="fp16_split")
    c = mck.fused_logits(plan, x, W, prec="fp16_split")
    assert torch.equal(a, c)


def test_unsupported(mck, dev):
    plan = mck.Plan(512, 2, "rbf", 3.0, 12)
    x = torch.zeros((4, 512), device=dev)
    W = torch.zeros((10, plan.num_features), device=dev)
    with pytest.raises(mck.MckError, match="UNSUPPORTED"):
        mck.fused_logits(plan, x, W, prec="fp16_split")
    p2 = mck.Plan(1024, 2, "rbf", 3.0, 12)
    W2 = torch.zeros((10, p2.num_features), device=dev)
    with pytest.raises(mck.MckError, match="UNSUPPORTED"):
        mck.fused_logits(p2, torch.zeros((4, 784), device=dev), W2, prec="bf16_split")
    # an empty batch is fine
    out = mck.fused_logits(p2, torch.zeros((0, 784), device=dev), W2, prec="fp16_split")
    assert out.shape == (0, 10)
