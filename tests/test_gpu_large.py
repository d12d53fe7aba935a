"""Dimensions past the fused kernels: features at 2^15 < d <= 2^20 and the
adjoint at 2^11 <= d <= 2^20 run in passes over HBM scratch, rows in chunks.

* Plans above 2^15 draw their permutations on the host: bit-exact against the
  oracle's Fisher-Yates.
* Features at d = 2^16..2^20 against the oracle at sampled output
  coordinates (output k uses the calibration only through C_e[k], so the
  oracle runs both transforms in full and computes C_e[k] for the sampled k).
  Per-coordinate bar: 1e-5 plus float32's resolution of the phase and the
  transform's rounding, 2^-24 (|z_k| + 4 log2(d) Cs_k max_j |h_j|).
* The adjoint at d = 2^11..2^16 and the fused logits with their gradients at
  2^16 against the oracle's chain rule (full tables): gradients within 1e-4
  of the largest oracle entry, logits within 1e-4.
* Row chunks: a batch spanning several scratch chunks gives the features of
  each row as alone, and batch sums equal to the sums over the chunks' rows.
"""

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import fastfood as ff
from oracle import training as tr

pytestmark = pytest.mark.gpu

_T = {}


def _tables(d, E, kernel, sigma, seed):
    key = (d, E, kernel, sigma, seed)
    if key not in _T:
        _T[key] = ff.plan_tables(d, E, kernel, sigma, seed=seed)
    return _T[key]


def _rel(got, ref):
    return float(np.abs(got.astype(np.float64) - ref).max() / max(np.abs(ref).max(), 1e-30))


def _radius(kernel, d, e, k, seed):
    return ff.laplace_radius(d, e, k, seed) if kernel == ff.LAPLACE else ff.rbf_radius(d, e, k, seed)


def _check_sampled(phi_rows, x, d, E, kernel, sigma, seed, nks=6):
    """phi_rows (n, 2Ed) of rows x (n, in_dim) against the oracle at sampled k."""
    B, perm, G = ff.table_B(d, E, seed), ff.table_perm(d, E, seed), ff.table_G(d, E, seed)
    gnorm = np.linalg.norm(G, axis=1)
    rng = np.random.default_rng(d + E)
    got = phi_rows.astype(np.float64).reshape(len(x), E, 2, d)
    for e in range(E):
        ks = np.unique(np.concatenate([[0, d - 1], rng.integers(0, d, nks)]))
        cs = np.array([_radius(kernel, d, e, int(k), seed) for k in ks]) / gnorm[e] / (sigma * np.sqrt(d))
        h = ff.stages(x.astype(np.float64), B[e], perm[e], G[e], np.ones(d))["h"]  # (n, d)
        z = cs[None] * h[:, ks]
        tol = 1e-5 + 2.0 ** -24 * (np.abs(z) + 4 * np.log2(d) * cs[None] * np.abs(h).max(axis=1, keepdims=True))
        assert np.all(np.abs(got[:, e, 0, ks] - np.cos(z)) <= tol), (d, e)
        assert np.all(np.abs(got[:, e, 1, ks] - np.sin(z)) <= tol), (d, e)


def test_host_permutation_matches_oracle(mck):
    d = 1 << 16
    plan = mck.Plan(d, 2, "rbf", 1.0, 77)
    np.testing.assert_array_equal(plan.tables()["perm"].astype(np.int64), ff.table_perm(d, 2, 77))
    plan.close()


@pytest.mark.parametrize("L,E,n,kernel", [(16, 2, 3, "rbf"), (17, 1, 2, "laplace"),
                                          (18, 1, 2, "rbf"), (20, 1, 2, "rbf")])
def test_large_d_features_sampled(mck, dev, L, E, n, kernel):
    d = 1 << L
    sigma, seed = 3.0, 100 + L
    plan = mck.Plan(d, E, kernel, sigma, seed)
    x = wl.mnist_like(n, 784, seed=L)
    phi = mck.features(plan, torch.from_numpy(x).to(dev)).cpu().numpy()
    assert phi.shape == (n, 2 * E * d) and np.isfinite(phi).all()
    _check_sampled(phi, x, d, E, ff.LAPLACE if kernel == "laplace" else ff.RBF, sigma, seed)
    plan.close()


def test_large_d_chunks_of_rows(mck, dev):
    """d = 2^16, E = 16: 32 rows per scratch chunk, so 70 rows run in three
    chunks; sampled rows of every chunk against the oracle and against the
    same rows computed alone."""
    d, E, n = 1 << 16, 16, 70
    plan = mck.Plan(d, E, "rbf", 3.0, 5)
    x = wl.mnist_like(n, 784, seed=9)
    xd = torch.from_numpy(x).to(dev)
    phi = mck.features(plan, xd)
    rows = [0, 31, 32, 63, 64, 69]
    for r in rows:
        assert torch.equal(phi[r], mck.features(plan, xd[r:r + 1])[0])
    # the first two expansions of rows from each chunk (a plan with E = 2 and
    # the same seed has the same first two expansions)
    sub = phi[[0, 40, 69]].view(3, E, 2 * d)[:, :2].reshape(3, 4 * d).cpu().numpy()
    _check_sampled(sub, x[[0, 40, 69]], d, 2, ff.RBF, 3.0, 5, nks=3)
    plan.close()


@pytest.mark.parametrize("d,E,n", [(2048, 2, 5), (1 << 13, 1, 3), (1 << 14, 2, 3), (1 << 16, 1, 2)])
def test_large_d_adjoint(mck, dev, d, E, n):
    sigma, seed = 3.0, 31
    plan = mck.Plan(d, E, "rbf", sigma, seed)
    x = wl.mnist_like(n, 784, seed=d)
    dphi = np.random.default_rng(d).standard_normal((n, 2 * E * d)).astype(np.float32)
    dx, dCs, dG, dB = mck.features_backward(plan, torch.from_numpy(x).to(dev),
                                            torch.from_numpy(dphi).to(dev), need_dB=True)
    rx, rCs, rG, rB = tr.features_backward(x.astype(np.float64), _tables(d, E, ff.RBF, sigma, seed),
                                           dphi.astype(np.float64), with_dB=True)
    for got, ref in ((dx, rx), (dCs, rCs), (dG, rG), (dB, rB)):
        assert _rel(got.cpu().numpy(), ref) <= 1e-4
    plan.close()


def test_large_d_fused_logits_and_gradients(mck, dev):
    d, E, n, C = 1 << 16, 1, 3, 10
    sigma, seed = 3.0, 31
    plan = mck.Plan(d, E, "rbf", sigma, seed)
    x = wl.mnist_like(n, 784, seed=d)
    W, _ = wl.logit_weights(C, 2 * E * d, seed=4, std=0.05)
    b = np.linspace(-1, 1, C).astype(np.float32)
    y = wl.labels(n, C, seed=2)
    xd, Wd, bd = (torch.from_numpy(a).to(dev) for a in (x, W, b))
    logits = mck.fused_logits(plan, xd, Wd, bd)
    _, dl = mck.softmax_xent(logits, torch.from_numpy(y).to(dev))
    g = mck.fused_logits_backward(plan, xd, Wd, dl, need_dx=True, need_dB=True)
    o = tr.train_grads(x.astype(np.float64), _tables(d, E, ff.RBF, sigma, seed),
                       W.astype(np.float64), b.astype(np.float64), y)
    assert np.abs(logits.cpu().numpy() - o["logits"]).max() <= 1e-4
    for k in ("dx", "dCs", "dG", "dB", "dW", "db"):
        assert _rel(g[k].cpu().numpy(), o[k]) <= 1e-4, k
    plan.close()


def test_adjoint_chunks_sum_like_their_rows(mck, dev):
    """d = 2^16, E = 16: 21 rows per adjoint chunk; 25 rows (two chunks) give
    dx row by row as the rows alone, and batch sums equal the sums of the two
    chunks' own sums (float32 reassociation only)."""
    d, E, n = 1 << 16, 16, 25
    plan = mck.Plan(d, E, "rbf", 3.0, 6)
    x = torch.from_numpy(wl.mnist_like(n, 784, seed=3)).to(dev)
    dphi = torch.from_numpy(np.random.default_rng(1).standard_normal((n, 2 * E * d)).astype(np.float32)).to(dev)
    full = mck.features_backward(plan, x, dphi, need_dB=True)
    a = mck.features_backward(plan, x[:21], dphi[:21], need_dB=True)
    b = mck.features_backward(plan, x[21:], dphi[21:], need_dB=True)
    assert torch.equal(full[0][:21], a[0]) and torch.equal(full[0][21:], b[0])
    for i in (1, 2, 3):
        ref = (a[i].double() + b[i].double())
        assert float((full[i].double() - ref).abs().max() / ref.abs().max()) <= 1e-6
    plan.close()
