"""Learned signs B (Sec. "Empirical Analysis": learning B, likened to
attention) against the FP64 oracle.

* mck_plan_set_signs: the plan's B becomes the signs of a real array, in
  every table layout (bit words, lane masks of the warp kernels, chunk masks
  of the block kernels), so features of every kernel family match the oracle
  run with the same B;
* dB, the gradient with respect to B read as a real diagonal, from
  mck_features_backward_ex and mck_fused_logits_backward_ex; requesting it
  leaves the other gradients unchanged (bit-identical, except dCs and dG of
  the fused adjoint at d = 1024, which are then summed in another order);
* the straight-through classifier: B.grad equals the gated oracle gradient.

Bars as for the other gradients: within 1e-4 of the largest oracle entry.
"""

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import fastfood as ff
from oracle import training as tr

pytestmark = pytest.mark.gpu


def _tables(plan, B=None):
    T = ff.plan_tables(plan.d, plan.E, plan.kernel, plan.sigma, t=plan.matern_t or 40,
                       seed=plan.seed)
    if B is not None:
        T["B"] = np.where(B < 0, -1.0, 1.0)
    return T


def _rel(got, ref):
    return float(np.abs(got.astype(np.float64) - ref).max() / max(np.abs(ref).max(), 1e-30))


def _tables32(plan, B=None):
    """The oracle's tables with Cs rounded to float32, the precision the
    library stores it in (held to one float32 ulp of the oracle by the table
    tests)."""
    T = _tables(plan, B)
    T["Cs"] = T["Cs"].astype(np.float32).astype(np.float64)
    return T


def _phase_tol(z, Cs, d):
    """Per-feature bound of a float32 feature against the float64 oracle run
    on float32-rounded Cs, (n, 2 E d): 1e-5 plus float32's resolution of the
    phase and the transform's rounding, 2^-24 (|z_k| + 4 log2(d) Cs_k max|h|).
    Needed for Laplacian plans, whose heavy-tailed radii give a few large
    phases; capped at 2 (any value in [-1, 1] passes)."""
    Cs = Cs[None]
    hmax = np.abs(z / Cs).max(axis=2, keepdims=True)
    t = 1e-5 + 2.0 ** -24 * (np.abs(z) + 4 * np.log2(d) * Cs * hmax)
    return np.minimum(np.concatenate([t, t], axis=2).reshape(z.shape[0], -1), 2.0)


def _latent(E, d, seed):
    g = np.random.default_rng(seed)
    B = g.standard_normal((E, d)).astype(np.float32)
    B[0, :3] = [0.0, -0.0, np.float32(-1e-30)]  # 0 and -0 give +1, a tiny negative -1
    return B


@pytest.mark.parametrize("d,E,n", [(8, 2, 5), (64, 3, 7), (1024, 2, 9), (4096, 2, 3),
                                   (1 << 15, 1, 2)])
def test_set_signs_features(mck, dev, d, E, n):
    plan = mck.Plan(d, E, "rbf", 2.0, 77)
    B = _latent(E, d, seed=d)
    plan.set_signs(torch.from_numpy(B).to(dev))
    want = np.where(B < 0, -1.0, 1.0)
    want[0, 1] = 1.0  # -0.0 is not < 0
    np.testing.assert_array_equal(plan.signs(), want)
    in_dim = min(d, 784)
    x = (wl.gaussian(n, in_dim, seed=n) * np.float32(6 * 2.0 / np.sqrt(in_dim))).astype(np.float32)
    phi = mck.features(plan, torch.from_numpy(x).to(dev)).cpu().numpy()
    ref = ff.features(x.astype(np.float64), _tables(plan, B))
    assert float(np.abs(phi.astype(np.float64) - ref).max()) <= 1e-5
    # the tables other than B are untouched
    t0 = ff.plan_tables(d, E, ff.RBF, 2.0, seed=77)
    np.testing.assert_array_equal(plan.tables()["perm"].astype(np.int64), t0["perm"])
    plan.close()


@pytest.mark.parametrize("d,E,n,in_dim", [(32, 2, 5, 32), (64, 2, 19, 50), (256, 3, 8, 256),
                                          (1024, 2, 9, 784), (1024, 1, 40, 1024)])
def test_features_backward_dB(mck, dev, d, E, n, in_dim):
    plan = mck.Plan(d, E, "rbf", 1.0, 21)
    B = _latent(E, d, seed=d + 1)
    plan.set_signs(torch.from_numpy(B).to(dev))
    x = wl.mnist_like(n, in_dim, seed=d)
    dphi = np.random.default_rng(5).standard_normal((n, plan.num_features)).astype(np.float32)
    xd, dpd = torch.from_numpy(x).to(dev), torch.from_numpy(dphi).to(dev)
    dx, dCs, dG, dB = mck.features_backward(plan, xd, dpd, need_dB=True)
    rx, rc, rg, rb = tr.features_backward(x.astype(np.float64), _tables(plan, B),
                                          dphi.astype(np.float64), with_dB=True)
    assert _rel(dB.cpu().numpy(), rb) <= 1e-4
    assert torch.all(dB[:, in_dim:] == 0)
    assert _rel(dCs.cpu().numpy(), rc) <= 1e-4 and _rel(dG.cpu().numpy(), rg) <= 1e-4
    # asking for dB changes nothing else (same sums in the same order)
    dx2, dCs2, dG2 = mck.features_backward(plan, xd, dpd)
    assert torch.equal(dx, dx2) and torch.equal(dCs, dCs2) and torch.equal(dG, dG2)
    # dB alone
    only = mck.features_backward(plan, xd, dpd, need_dx=False, need_dCs=False, need_dG=False,
                                 need_dB=True)[3]
    assert torch.equal(only, dB)
    plan.close()


@pytest.mark.parametrize("d,E,C,n", [(64, 2, 3, 9), (256, 2, 10, 33), (1024, 2, 10, 17),
                                     (1024, 4, 16, 70)])
def test_fused_logits_backward_dB(mck, dev, d, E, C, n):
    plan = mck.Plan(d, E, "rbf", 1.0, 5)
    B = _latent(E, d, seed=3 * d)
    plan.set_signs(torch.from_numpy(B).to(dev))
    x = wl.mnist_like(n, min(d, 784), seed=d)
    W, _ = wl.logit_weights(C, 2 * E * d, seed=1, std=0.05)
    dl = (np.random.default_rng(9).standard_normal((n, C)) * 0.1).astype(np.float32)
    xd, Wd, dld = (torch.from_numpy(a).to(dev) for a in (x, W, dl))
    g = mck.fused_logits_backward(plan, xd, Wd, dld, need_dx=True, need_dB=True)
    T = _tables(plan, B)
    phi = ff.features(x.astype(np.float64), T)
    _, _, _, rb = tr.features_backward(x.astype(np.float64), T, dl.astype(np.float64) @ W,
                                       with_dB=True)
    assert _rel(g["dB"].cpu().numpy(), rb) <= 1e-4
    assert _rel(g["dW"].cpu().numpy(), dl.T.astype(np.float64) @ phi) <= 1e-4
    g2 = mck.fused_logits_backward(plan, xd, Wd, dld, need_dx=True)
    # dx, dW and db come from the same launches either way; at d = 1024 the
    # row-tile path of the parameter kernel (dphi formed for 8 rows at a time
    # in shared memory) has no room left for the dB sums, so dCs and dG are
    # then summed in another sample order: equal to rounding
    for k in ("dx", "dW", "db"):
        assert torch.equal(g[k], g2[k]), k
    for k in ("dCs", "dG"):
        if d < 1024:
            assert torch.equal(g[k], g2[k]), k
        else:
            ref = g2[k].abs().max().item()
            assert (g[k] - g2[k]).abs().max().item() <= 1e-5 * ref, k
    assert g2["dB"] is None
    plan.close()


def test_classifier_straight_through_signs(mck, dev):
    from paper_1702_08159_gb300.autograd import McKernelClassifier

    d, E, C, n = 256, 2, 10, 64
    plan = mck.Plan(d, E, "rbf", 2.0, 13)
    W, b = wl.logit_weights(C, 2 * E * d, seed=4, std=0.05)
    model = McKernelClassifier(plan, C, W=torch.from_numpy(W), b=torch.from_numpy(b),
                               learn_signs=True)
    with torch.no_grad():  # latents: some past the gate, some negative, one exactly 0
        Br = torch.from_numpy(_latent(E, d, seed=2)).to(dev) * 1.5
        model.Br.copy_(Br)
    x = wl.mnist_like(n, 200, seed=6)
    y = wl.labels(n, C, seed=6)
    loss = model.loss(torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev))
    loss.backward()
    Bl = Br.cpu().numpy()
    T = _tables(plan, Bl)
    g = tr.train_grads(x.astype(np.float64), T, W.astype(np.float64), b.astype(np.float64), y)
    assert abs(loss.item() - g["loss"]) <= 1e-5
    ref = g["dB"] * (np.abs(Bl) <= 1)
    assert _rel(model.Br.grad.cpu().numpy(), ref) <= 1e-4
    assert torch.all(model.Br.grad[Br.abs() > 1] == 0)
    # a step that flips signs changes the plan's B at the next forward
    with torch.no_grad():
        model.Br.copy_(-model.Br)
    model(torch.from_numpy(x[:2]).to(dev))
    np.testing.assert_array_equal(plan.signs(), np.where(-Bl < 0, -1.0, 1.0))
    plan.close()


def test_group_sees_new_signs_and_laplace_plans(mck, dev):
    """A group built before mck_plan_set_signs uses the new signs (it reads the
    plans' tables at launch), including the lane and chunk masks of its warp
    steps and block items; one of the plans has the Laplacian calibration."""
    specs = [(64, "rbf"), (1024, "laplace"), (4096, "rbf")]
    plans = [mck.Plan(d, 3, k, 3.0, 99) for d, k in specs]
    Bs = [_latent(3, d, seed=500 + d) for d, _ in specs]
    E = [3, 2, 3, 1, 2, 3]
    pidx = [0, 1, 2, 0, 1, 2]
    in_dims = [64, 784, 4000, 60, 1024, 4096]
    items, x_len, phi_len = mck.group_layout(plans, pidx, E, in_dims)
    xh = np.zeros(x_len, np.float32)
    xs = []
    for i, n in enumerate(in_dims):
        v = (wl.gaussian(1, n, seed=i)[0] * np.float32(6.0 / np.sqrt(n))).astype(np.float32)
        xh[items["x_offset"][i]: items["x_offset"][i] + n] = v
        xs.append(v)
    group = mck.Group(plans, items, x_len, phi_len)
    for p, B in zip(plans, Bs):
        p.set_signs(torch.from_numpy(B).to(dev))
    x = torch.from_numpy(xh).to(dev)
    phi = torch.full((phi_len,), float("nan"), device=dev)
    group.features(x, phi)
    got = phi.cpu().numpy().astype(np.float64)
    for i, (p, e, n) in enumerate(zip(pidx, E, in_dims)):
        plan = plans[p]
        T = _tables32(plan, Bs[p])
        Te = {k: (v[:e] if isinstance(v, np.ndarray) else v) for k, v in T.items()}
        xi = xs[i][None].astype(np.float64)
        ref = ff.features(xi, Te)[0]
        tol = _phase_tol(ff.phases(xi, Te), Te["Cs"], plan.d)[0]
        o = int(items["phi_offset"][i])
        assert np.all(np.abs(got[o: o + 2 * e * plan.d] - ref) <= tol), i
    for p in plans:
        p.close()


def test_laplace_fused_logits(mck, dev):
    plan = mck.Plan(1024, 4, "laplace", 3.0, 31)
    x = wl.mnist_like(40, 784, seed=3)
    W, _ = wl.logit_weights(10, plan.num_features, seed=2, std=0.05)
    b = np.linspace(-1, 1, 10).astype(np.float32)
    got = mck.fused_logits(plan, torch.from_numpy(x).to(dev), torch.from_numpy(W).to(dev),
                           torch.from_numpy(b).to(dev)).cpu().numpy()
    # The oracle on its own float32-rounded Cs. Laplacian radii are heavy tailed,
    # so a few phases are large: each feature's float32 error is bounded as in
    # the Laplacian feature test, 2^-24 (|z_k| + 4 log2(d) Cs_k max_j |h_j|),
    # and the logits bar adds those bounds weighted by |W|.
    T = _tables32(plan)
    ft = _phase_tol(ff.phases(x.astype(np.float64), T), T["Cs"], plan.d)
    bar = 1e-4 + ft @ np.abs(W.astype(np.float64)).T
    ref = tr.logits(ff.features(x.astype(np.float64), T), W.astype(np.float64),
                    b.astype(np.float64))
    assert np.all(np.abs(got - ref) <= bar)
    assert np.abs(got - ref).max() <= 1e-3
    plan.close()
