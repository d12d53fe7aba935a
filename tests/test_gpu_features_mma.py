"""Tensor-core feature kernel (mck_features_ex, d = 1024) against the FP64 oracle.

Error model (the transform's, as in test_gpu_fwht_mma.py): each form's H
has max error eps * sqrt(d) rms(input) with eps = 2^-6, 2^-8, 2^-14, 2^-18
for bf16, fp16, bf16 hi/lo, fp16 hi/lo (factors 4-8 over the measured).
Both transforms feed the phase z = Cs h; the first one's error reaches h
through G and the second transform, so a feature (cos and sin are
1-Lipschitz) is off by at most
    2 eps Cs_k sqrt(d) rms(G v)      (rms over the row's second-transform input)
plus the FP32 bar 1e-5 for everything else. Separately, fp16 hi/lo is held
to the FP32 features' own bar, 1e-5, on the MNIST-shaped workloads.

The data operand is scaled per row by powers of two to stay in fp16's range:
scaling x and sigma together leaves the features unchanged, so huge and tiny
inputs must give the same features.
"""

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import fastfood as ff

pytestmark = pytest.mark.gpu

EPS = {"bf16": 2.0 ** -6, "fp16": 2.0 ** -8, "bf16_split": 2.0 ** -14, "fp16_split": 2.0 ** -18}


def _bound(x, T, eps):
    """Per-feature bound (n, 2Ed) of the error model above."""
    d = T["B"].shape[1]
    out = []
    for e in range(T["B"].shape[0]):
        st = ff.stages(x.astype(np.float64), T["B"][e], T["perm"][e], T["G"][e], T["Cs"][e])
        rms = np.sqrt((st["w"] ** 2).mean(axis=1, keepdims=True))
        b = 1e-5 + 2 * eps * T["Cs"][e][None] * np.sqrt(d) * rms
        out.append(np.concatenate([b, b], axis=1))
    return np.concatenate(out, axis=1)


@pytest.mark.parametrize("prec", list(EPS))
def test_tensor_core_features_error_model(mck, dev, prec):
    plan = mck.Plan(1024, 3, "rbf", 3.0, 42)
    x = wl.mnist_like(37, 784, seed=5)  # a ragged last tile of the 4-row items
    T = ff.plan_tables(1024, 3, ff.RBF, 3.0, seed=42)
    got = mck.features(plan, torch.from_numpy(x).to(dev), prec=prec).cpu().numpy()
    ref = ff.features(x.astype(np.float64), T)
    assert np.isfinite(got).all()
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= _bound(x, T, EPS[prec])), (prec, float(err.max()))
    plan.close()


@pytest.mark.parametrize("E,sigma,n,seed", [(16, 3.0, 300, 42), (8, 3.0, 64, 7), (1, 1.0, 256, 42)])
def test_fp16_split_meets_the_fp32_bar(mck, dev, E, sigma, n, seed):
    """MNIST-shaped rows (the headline, config 1 and config 0 shapes)."""
    plan = mck.Plan(1024, E, "rbf", sigma, seed)
    x = wl.mnist_like(n, 784, seed=seed + 1)
    rows = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(n).integers(0, n, 12)]))
    got = mck.features(plan, torch.from_numpy(x).to(dev), prec="fp16_split").cpu().numpy()
    ref = ff.features(x[rows].astype(np.float64), ff.plan_tables(1024, E, ff.RBF, sigma, seed=seed))
    assert float(np.abs(got[rows] - ref).max()) <= 1e-5
    plan.close()


@pytest.mark.parametrize("c", [1e5, 1e-5])
def test_row_scaling_keeps_huge_and_tiny_inputs(mck, dev, c):
    """(x, sigma) -> (c x, c sigma) leaves z = Cs h, hence the features,
    unchanged; without the per-row scaling c = 1e5 overflows fp16."""
    x = wl.mnist_like(9, 784, seed=3)
    T = ff.plan_tables(1024, 2, ff.RBF, 3.0, seed=11)
    ref = ff.features(x.astype(np.float64), T)
    plan = mck.Plan(1024, 2, "rbf", 3.0 * c, 11)
    got = mck.features(plan, torch.from_numpy((x * c).astype(np.float32)).to(dev),
                       prec="fp16_split").cpu().numpy()
    assert np.isfinite(got).all()
    assert np.all(np.abs(got - ref) <= _bound(x, T, EPS["fp16_split"]) + 1e-6)
    plan.close()


def test_tensor_core_features_with_learned_tables(mck, dev):
    """Caller-supplied Cs and G (natural order) instead of the plan's lane-ordered copies."""
    plan = mck.Plan(1024, 2, "rbf", 3.0, 9)
    T = ff.plan_tables(1024, 2, ff.RBF, 3.0, seed=9)
    g = np.random.default_rng(0)
    Cs = (T["Cs"] * (1 + 0.1 * g.standard_normal(T["Cs"].shape))).astype(np.float32)
    G = (T["G"] * (1 + 0.1 * g.standard_normal(T["G"].shape))).astype(np.float32)
    x = wl.mnist_like(11, 784, seed=9)
    got = mck.features(plan, torch.from_numpy(x).to(dev), torch.from_numpy(Cs).to(dev),
                       torch.from_numpy(G).to(dev), prec="fp16_split").cpu().numpy()
    T2 = dict(T, Cs=Cs.astype(np.float64), G=G.astype(np.float64))
    ref = ff.features(x.astype(np.float64), T2)
    assert np.all(np.abs(got - ref) <= _bound(x, T2, EPS["fp16_split"]))
    plan.close()


def test_tensor_core_features_need_d1024(mck, dev):
    plan = mck.Plan(512, 1, "rbf", 1.0, 1)
    with pytest.raises(mck.MckError, match="UNSUPPORTED"):
        mck.features(plan, torch.zeros((2, 512), device=dev), prec="fp16_split")
    plan.close()
