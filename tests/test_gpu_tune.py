"""Launch-shape tunables and the autotuner (GPU).

Every launch shape of the batched feature kernels and every regime of the
2^16 / 2^17 transform must give the same bits: the shapes only change how
work is split (rows per work item, shared-memory staging, cluster size), not
the arithmetic. Each shape is also held to the oracle directly. The tuner
must choose among several shapes, set the winner on the plan, and reuse its
JSON cache without timing again.
"""

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import fastfood as ff
from paper_1702_08159_gb300 import tune

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,E,n", [(64, 3, 67), (512, 2, 33), (1024, 3, 45), (2048, 3, 9),
                                   (4096, 2, 7), (1 << 13, 2, 5), (1 << 14, 2, 5)])
def test_every_launch_shape_gives_the_same_features(mck, dev, d, E, n):
    plan = mck.Plan(d, E, "rbf", 3.0, 17 + d)
    x = wl.mnist_like(n, min(d, 784), seed=d)
    xd = torch.from_numpy(x).to(dev)
    shapes = plan.launch_candidates()
    assert len(shapes) >= (2 if d >= 512 else 1)  # below 512 a warp round already holds >= 4 rows
    outs = []
    for shape in shapes:
        plan.set_launch(*shape)
        assert plan.launch() == shape
        outs.append(mck.features(plan, xd))
    plan.set_launch(0, -1)
    outs.append(mck.features(plan, xd))
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    rows = [0, n - 1]
    ref = ff.features(x[rows].astype(np.float64),
                      ff.plan_tables(d, E, ff.RBF, 3.0, seed=17 + d))
    assert float(np.abs(outs[0][rows].cpu().numpy() - ref).max()) <= 1e-5
    plan.close()


def test_unaligned_rows_with_staging_asked_for(mck, dev):
    """staged = 1 with rows that are not 16-byte aligned runs the unstaged
    kernel: same results."""
    d = 1 << 14
    plan = mck.Plan(d, 2, "rbf", 3.0, 5)
    x = torch.from_numpy(wl.mnist_like(6, 1001, seed=1)).to(dev)[:, 1:]  # in_dim 1000, odd offset
    ref = mck.features(plan, x.contiguous())
    plan.set_launch(2, 1)
    assert torch.equal(mck.features(plan, x), ref)
    plan.close()


def test_set_launch_rejects_other_shapes(mck):
    p = mck.Plan(1024, 1, "rbf", 1.0, 1)
    for bad in [(3, -1), (2, -1), (4, 0), (0, 2)]:
        with pytest.raises(mck.MckError, match="INVAL"):
            p.set_launch(*bad)
    q = mck.Plan(1 << 15, 1, "rbf", 1.0, 1)
    with pytest.raises(mck.MckError, match="INVAL"):
        q.set_launch(1, -1)
    q.set_launch(0, -1)
    p.close()
    q.close()


def test_tuner_chooses_sets_and_caches(mck, dev, tmp_path):
    cache = str(tmp_path / "tune.json")
    plan = mck.Plan(2048, 4, "rbf", 3.0, 42)
    x = torch.from_numpy(wl.mnist_like(512, 784, seed=3)).to(dev)
    best, times, cached = tune.tune_features(plan, x, reps=2, cache=cache)
    assert not cached and len(times) == 6 and best in times
    assert plan.launch() == best
    plan.set_launch(0, -1)
    best2, times2, cached2 = tune.tune_features(plan, x, reps=2, cache=cache)
    assert cached2 and best2 == best and plan.launch() == best
    assert set(times2) == set(times)
    plan.close()


@pytest.mark.parametrize("L", [16, 17])
def test_transform_regimes_agree(mck, dev, L, tmp_path):
    d = 1 << L
    x = wl.gaussian(3, d, seed=L)
    outs = []
    for regime in ("auto",) + tune.FWHT_REGIMES:
        t = torch.from_numpy(x).to(dev)
        mck.fwht_(t, "fp32", regime)
        outs.append(t)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    ref = ff.fwht(x.astype(np.float64))
    scale = np.sqrt(d) * np.sqrt((x.astype(np.float64) ** 2).mean())
    assert float(np.abs(outs[0].cpu().numpy() - ref).max()) / scale <= L * 2.0 ** -21
    cache = str(tmp_path / "t.json")
    w = torch.from_numpy(x).to(dev)
    r, ms, cached = tune.tune_fwht(w, reps=2, cache=cache)
    assert r in tune.FWHT_REGIMES and len(ms) == 3 and not cached
    r2, _, cached2 = tune.tune_fwht(w, reps=2, cache=cache)
    assert cached2 and r2 == r
    with pytest.raises(mck.MckError, match="INVAL"):
        mck.fwht_(torch.zeros((1, 1024), device=dev), "fp32", "two_pass")


def test_logit_contraction_tuner(mck, dev, tmp_path):
    """tune_logits times both contractions (each held to the fused logits'
    1e-4 bar against the oracle by tests/test_gpu_logits_mma.py), returns the
    faster one, and reuses its cache; at d != 1024 only FP32 exists."""
    cache = str(tmp_path / "tl.json")
    plan = mck.Plan(1024, 4, "rbf", 3.0, 42)
    x = torch.from_numpy(wl.mnist_like(3000, 784, seed=4)).to(dev)
    W = torch.from_numpy(wl.logit_weights(10, plan.num_features, seed=4)[0]).to(dev)
    prec, times, cached = tune.tune_logits(plan, x, W, reps=2, cache=cache)
    assert not cached and set(times) == set(tune.LOGIT_PRECISIONS) and prec in times
    assert times[prec] == min(times.values())
    prec2, times2, cached2 = tune.tune_logits(plan, x, W, reps=2, cache=cache)
    assert cached2 and prec2 == prec and set(times2) == set(times)
    a = mck.fused_logits(plan, x, W, prec=prec)
    b = mck.fused_logits(plan, x, W)
    assert (a - b).abs().max().item() <= 1e-4
    plan.close()
    p2 = mck.Plan(512, 2, "rbf", 3.0, 1)
    W2 = torch.zeros((10, p2.num_features), device=dev)
    assert tune.tune_logits(p2, torch.zeros((4, 512), device=dev), W2, cache=cache) == ("fp32", {}, False)
    p2.close()
