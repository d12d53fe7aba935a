"""The benchmark workloads at full size, in the launch configurations the bench
times, checked against the FP64 oracle on sampled outputs.

* config 1 (60000 MNIST-shaped rows, d = 1024, E = 8, sigma = 3, W ~ N(0, 0.01),
  b = 0): fused logits with RBF and Matern (t = 40) calibration, and the
  Matern features;
* the headline (E = 16): fused logits;
* config 4 (10000 vectors, d = 2^6..2^14, E = 1..32, RBF and Matern): the
  persistent grouped launch and its CUDA-graph replay.

Oracle tables are built only for the sampled outputs' plans and expansions:
the Matern calibration costs t d^2 draws per expansion on the CPU (about 4 s at
d = 1024) and the RBF radius one rejection loop per entry, so whole tables are
built only for small d and few expansions. Larger vectors (Matern above
d = 256, RBF with E > 24 above d = 1024) are checked at sampled output
coordinates: each output k of expansion e depends on the calibration only
through C_e[k], so the oracle runs both transforms with its own B, Pi and G
and computes C_e[k] for the sampled k alone.
Bars: features 1e-5 max abs error; logits 1e-4 (sums of 2 E d products).
"""

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import fastfood as ff
from oracle import training as tr

pytestmark = pytest.mark.gpu

N, IN_DIM, D, C = 60000, 784, 1024, 10
_TABLES = {}


def _tables(d, E, kernel, sigma, seed, t=40):
    key = (d, E, kernel, sigma, seed, t)
    if key not in _TABLES:
        _TABLES[key] = ff.plan_tables(d, E, kernel, sigma, t=t, seed=seed)
    return _TABLES[key]


def _rows(n, seed=0, extra=25):
    return np.unique(np.concatenate([[0, 1, 7, 8, n // 2, n - 2, n - 1],
                                     np.random.default_rng(seed).integers(0, n, extra)]))


@pytest.fixture(scope="module")
def mnist(dev):
    x = wl.mnist_like(N, IN_DIM, seed=42)
    return x, torch.from_numpy(x).to(dev)


@pytest.mark.parametrize("E,kernel", [(8, "rbf"), (8, "matern"), (16, "rbf")])
def test_fused_logits_full_size_sampled(mck, dev, mnist, E, kernel):
    x, xd = mnist
    plan = mck.Plan(D, E, kernel, 3.0, 42, matern_t=40)
    W, b = wl.logit_weights(C, plan.num_features, seed=42)
    got = mck.fused_logits(plan, xd, torch.from_numpy(W).to(dev),
                           torch.from_numpy(b).to(dev)).cpu().numpy()
    rows = _rows(N)
    T = _tables(D, E, ff.RBF if kernel == "rbf" else ff.MATERN, 3.0, 42)
    ref = tr.logits(ff.features(x[rows].astype(np.float64), T), W.astype(np.float64),
                    b.astype(np.float64))
    assert np.abs(got[rows] - ref).max() <= 1e-4
    assert np.isfinite(got).all()
    plan.close()


def test_config1_matern_features_full_size_sampled(mck, dev, mnist):
    x, xd = mnist
    plan = mck.Plan(D, 8, "matern", 3.0, 42, matern_t=40)
    phi = mck.features(plan, xd)
    rows = _rows(N, seed=1)
    got = phi[torch.from_numpy(rows).to(dev)].cpu().numpy()
    del phi
    torch.cuda.empty_cache()
    ref = ff.features(x[rows].astype(np.float64), _tables(D, 8, ff.MATERN, 3.0, 42))
    assert float(np.abs(got.astype(np.float64) - ref).max()) <= 1e-5
    plan.close()


def _oracle_at(xi, d, E, kernel, sigma, seed, ks, t=40):
    """Oracle features of one vector at output coordinates ks (per expansion
    e, a list of k) for expansions 0..E-1: both transforms in full with the
    oracle's B, Pi and G, the calibration only at the sampled k. Returns
    per-expansion (cos, sin, z, Cs at ks, max_j |h_j|)."""
    B = ff.table_B(d, E, seed)
    perm = ff.table_perm(d, E, seed)
    G = ff.table_G(d, E, seed)
    gnorm = np.linalg.norm(G, axis=1)
    out = []
    for e in range(E):
        h = ff.stages(xi, B[e], perm[e], G[e], np.ones(d))["h"][0]
        if kernel == ff.MATERN:
            r = np.array([ff.ball_sum_norm(d, e, k, t, seed) for k in ks[e]])
        else:
            r = np.array([ff.rbf_radius(d, e, k, seed) for k in ks[e]])
        cs = r / gnorm[e] / (sigma * np.sqrt(d))
        z = cs * h[ks[e]]
        out.append((np.cos(z), np.sin(z), z, cs, float(np.abs(h).max())))
    return out


def test_config4_large_vectors_sampled(mck, dev):
    """The uneven batch's Matern vectors at d = 2^9..2^14 (largest and
    smallest E at each d) and its RBF vectors with E > 24 at d = 2^11..2^14,
    at sampled coordinates of every expansion, against the oracle alone.
    Per-coordinate bar: 1e-5 plus float32's resolution of the phase and the
    transform's rounding, 2^-24 (|z_k| + 4 log2(d) C_k max_j |h_j|) (phases
    reach hundreds with N(0,1) entries and sigma = 1)."""
    b = wl.uneven_batch(10000, seed=42)
    keys = sorted(set(zip(b["d"].tolist(), b["kernel"].tolist())))
    plans = [mck.Plan(d, 32, "rbf" if k == 0 else "matern", 1.0, 42, matern_t=40)
             for d, k in keys]
    pidx = np.array([keys.index((d, k)) for d, k in zip(b["d"].tolist(), b["kernel"].tolist())])
    order = np.lexsort((b["E"], b["kernel"], b["d"]))
    items, x_len, phi_len = mck.group_layout(plans, pidx, b["E"], b["d"], order)
    xh = np.zeros(x_len, np.float32)
    for i, v in enumerate(b["x"]):
        xh[items["x_offset"][i]: items["x_offset"][i] + len(v)] = v
    g = mck.Group(plans, items, x_len, phi_len)
    phi = torch.full((phi_len,), float("nan"), device=dev)
    g.features(torch.from_numpy(xh).to(dev), phi)
    torch.cuda.synchronize()
    picks = []
    for L in range(9, 15):
        d = 1 << L
        mat = np.nonzero((b["d"] == d) & (b["kernel"] == 1))[0]
        if len(mat):
            picks.append(int(mat[np.argmax(b["E"][mat])]))
            picks.append(int(mat[np.argmin(b["E"][mat])]))
        if L >= 11:
            rbf = np.nonzero((b["d"] == d) & (b["kernel"] == 0) & (b["E"] > 24))[0]
            if len(rbf):
                picks.append(int(rbf[np.argmax(b["E"][rbf])]))
    assert len(picks) >= 14
    assert max(int(b["E"][i]) for i in picks if b["kernel"][i] == 1 and b["d"][i] >= 4096) > 24
    rng = np.random.default_rng(7)
    for i in sorted(set(picks)):
        d, E, kern = int(b["d"][i]), int(b["E"][i]), int(b["kernel"][i])
        ks = [sorted({0, d - 1, int(rng.integers(0, d))}) for _ in range(E)]
        ref = _oracle_at(b["x"][i][None].astype(np.float64), d, E,
                         ff.RBF if kern == 0 else ff.MATERN, 1.0, 42, ks)
        o = int(items["phi_offset"][i])
        got = phi[o: o + 2 * E * d].cpu().numpy().astype(np.float64).reshape(E, 2, d)
        for e, (c, s_, z, cs, hmax) in enumerate(ref):
            tol = 1e-5 + 2.0 ** -24 * (np.abs(z) + 4 * np.log2(d) * cs * hmax)
            err_c = np.abs(got[e, 0, ks[e]] - c)
            err_s = np.abs(got[e, 1, ks[e]] - s_)
            assert np.all(err_c <= tol) and np.all(err_s <= tol), \
                (i, d, E, kern, e, float(err_c.max()), float(err_s.max()), tol)
    for p in plans:
        p.close()


def test_config4_full_size_sampled(mck, dev):
    """The bench's uneven batch: plans keyed by (d, kernel) with 32 expansions,
    packed in (d, kernel, E) order; sampled vectors against the oracle, and the
    graph replay identical to the direct launch."""
    b = wl.uneven_batch(10000, seed=42)
    keys = sorted(set(zip(b["d"].tolist(), b["kernel"].tolist())))
    plans = [mck.Plan(d, 32, "rbf" if k == 0 else "matern", 1.0, 42, matern_t=40)
             for d, k in keys]
    pidx = np.array([keys.index((d, k)) for d, k in zip(b["d"].tolist(), b["kernel"].tolist())])
    order = np.lexsort((b["E"], b["kernel"], b["d"]))
    items, x_len, phi_len = mck.group_layout(plans, pidx, b["E"], b["d"], order)
    xh = np.zeros(x_len, np.float32)
    for i, v in enumerate(b["x"]):
        xh[items["x_offset"][i]: items["x_offset"][i] + len(v)] = v
    x = torch.from_numpy(xh).to(dev)
    g = mck.Group(plans, items, x_len, phi_len)
    phi = torch.full((phi_len,), float("nan"), device=dev)
    g.features(x, phi)
    cap = mck.CapturedGroup(g, x, phi)
    phi2 = phi.clone()
    phi.fill_(float("nan"))
    cap.replay()
    torch.cuda.synchronize()
    assert torch.equal(phi, phi2)
    # samples: per d, the first RBF vector with E <= 6 and the last RBF vector
    # with E > 24 at d <= 1024; Matern vectors at d <= 256 with E <= 3
    picks = []
    for L in range(6, 15):
        d = 1 << L
        rbf = np.nonzero((b["d"] == d) & (b["kernel"] == 0))[0]
        small = rbf[b["E"][rbf] <= 6]
        if len(small):
            picks.append(int(small[0]))
        big = rbf[b["E"][rbf] > 24]
        if d <= 1024 and len(big):
            picks.append(int(big[-1]))
        if d <= 256:
            mat = np.nonzero((b["d"] == d) & (b["kernel"] == 1) & (b["E"] <= 3))[0]
            if len(mat):
                picks.append(int(mat[0]))
    assert len(picks) >= 12
    for i in picks:
        d, E, kern = int(b["d"][i]), int(b["E"][i]), int(b["kernel"][i])
        T = _tables(d, E, ff.RBF if kern == 0 else ff.MATERN, 1.0, 42)
        xi = b["x"][i][None].astype(np.float64)
        z = ff.phases(xi, T)
        ref = np.concatenate([np.cos(z), np.sin(z)], axis=2).reshape(-1)
        o = int(items["phi_offset"][i])
        got = phi[o: o + 2 * E * d].cpu().numpy().astype(np.float64)
        # With N(0,1) entries and sigma = 1 the phases reach |z| ~ 4 sqrt(d)
        # (hundreds at d = 2^14), which float32 itself resolves only to
        # |z| 2^-24: the bar adds log2(d) roundings of the largest phase.
        tol = 1e-5 + np.log2(d) * 2.0 ** -24 * float(np.abs(z).max())
        assert np.abs(got - ref).max() <= tol, (i, d, E, kern, float(np.abs(got - ref).max()), tol)
    for p in plans:
        p.close()
