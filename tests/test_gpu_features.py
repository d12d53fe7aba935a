"""Fused feature kernel (mck_features) against the FP64 oracle.

Bar: max abs error <= 1e-5 on every feature (float32 path vs float64 oracle).
Sizes span the three kernels (thread: d <= 16, warp: 32 <= d <= 1024, block:
2048 <= d <= 32768), ragged batches, ragged and strided inputs, learned
(overridden) C and G, both calibrations, and the full-size workloads on
sampled rows.
"""

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import fastfood as ff

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _oracle_tables(plan):
    return ff.plan_tables(plan.d, plan.E, plan.kernel, plan.sigma, t=plan.matern_t or 40,
                          seed=plan.seed)


def _max_err(got, ref):
    return float(np.abs(got.astype(np.float64) - ref).max())


def test_config0_full(mck, dev):
    # N=256 MNIST-shaped rows (784 -> 1024), E=1, sigma=1, RBF, seed 42.
    plan = mck.Plan(1024, 1, "rbf", 1.0, 42)
    x = wl.mnist_like(256, 784, seed=42)
    phi = mck.features(plan, torch.from_numpy(x).to(dev)).cpu().numpy()
    assert phi.shape == (256, 2048)
    ref = ff.features(x.astype(np.float64), _oracle_tables(plan))
    assert _max_err(phi, ref) <= TOL


@pytest.mark.parametrize("L", list(range(1, 16)))
def test_all_sizes(mck, dev, L):
    d = 1 << L
    E = 2 if L < 14 else 1
    n = 9 if L <= 12 else 3
    plan = mck.Plan(d, E, "rbf", 2.0, 1000 + L)
    in_dim = max(1, d - d // 4)
    # ||x|| ~ 6 sigma at every d, as for the MNIST-shaped rows (phases |z| up to ~30).
    # Much larger phases cannot meet 1e-5 in any float32 path: the spacing of
    # float32 numbers near |z| = 128 is already 1.5e-5.
    x = (wl.gaussian(n, in_dim, seed=L) * np.float32(6 * 2.0 / np.sqrt(in_dim))).astype(np.float32)
    phi = mck.features(plan, torch.from_numpy(x).to(dev)).cpu().numpy()
    ref = ff.features(x.astype(np.float64), _oracle_tables(plan))
    assert _max_err(phi, ref) <= TOL


@pytest.mark.parametrize("d,E,n,in_dim", [(2048, 3, 120, 1500), (16384, 2, 200, 12288),
                                          (16384, 3, 61, 16384)])
def test_chunked_blocks_take_several_items(mck, dev, d, E, n, in_dim):
    """More items than blocks, so every block runs several (row, expansion)
    items in turn; at d = 2^14 with 16-byte rows this is the staged kernel,
    which copies the next item's input and the current item's Cs into shared
    memory while the block works (zero-filled past in_dim)."""
    plan = mck.Plan(d, E, "rbf", 2.0, 4242 + d)
    x = (wl.gaussian(n, in_dim, seed=n) * np.float32(6 * 2.0 / np.sqrt(in_dim))).astype(np.float32)
    phi = mck.features(plan, torch.from_numpy(x).to(dev)).cpu().numpy()
    ref = ff.features(x.astype(np.float64), _oracle_tables(plan))
    assert _max_err(phi, ref) <= TOL
    plan.close()


@pytest.mark.parametrize("in_dim", [1, 3, 783, 784, 1024])
def test_ragged_input_dims(mck, dev, in_dim):
    plan = mck.Plan(1024, 2, "rbf", 1.0, 5)
    x = wl.mnist_like(17, in_dim, seed=in_dim)
    phi = mck.features(plan, torch.from_numpy(x).to(dev)).cpu().numpy()
    ref = ff.features(x.astype(np.float64), _oracle_tables(plan))
    assert _max_err(phi, ref) <= TOL


@pytest.mark.parametrize("n", [1, 2, 7, 8, 9, 31, 33])
def test_ragged_batches(mck, dev, n):
    for d in (32, 128, 1024):
        plan = mck.Plan(d, 3, "rbf", 1.0, 11)
        x = (wl.gaussian(n, d, seed=n) * np.float32(6 / np.sqrt(d))).astype(np.float32)
        phi = mck.features(plan, torch.from_numpy(x).to(dev)).cpu().numpy()
        ref = ff.features(x.astype(np.float64), _oracle_tables(plan))
        assert _max_err(phi, ref) <= TOL


@pytest.mark.parametrize("d,in_dim,ld", [(1024, 784, 900), (4096, 3001, 3100), (16384, 12000, 12345)])
def test_strided_and_misaligned_rows(mck, dev, d, in_dim, ld):
    plan = mck.Plan(d, 2, "rbf", 1.0, 13)
    base = (wl.mnist_like(6, ld, seed=3) * np.float32(np.sqrt(784 / in_dim))).astype(np.float32)
    t = torch.from_numpy(base).to(dev)
    ref_tab = _oracle_tables(plan)
    # rows with leading dimension ld > in_dim
    phi = mck.features(plan, t[:, :in_dim]).cpu().numpy()
    assert _max_err(phi, ff.features(base[:, :in_dim].astype(np.float64), ref_tab)) <= TOL
    # rows starting one float past a 16-byte boundary (scalar load path)
    phi = mck.features(plan, t[:, 1:in_dim + 1]).cpu().numpy()
    assert _max_err(phi, ff.features(base[:, 1:in_dim + 1].astype(np.float64), ref_tab)) <= TOL


def test_empty_batch(mck, dev):
    plan = mck.Plan(1024, 2, "rbf", 1.0, 1)
    out = mck.features(plan, torch.empty((0, 784), device=dev))
    assert out.shape == (0, 4096)


@pytest.mark.parametrize("d", [8, 256, 1024, 4096])
def test_overridden_calibration_and_gaussian(mck, dev, d):
    plan = mck.Plan(d, 2, "rbf", 1.0, 17)
    T = _oracle_tables(plan)
    g = np.random.default_rng(d)
    Cs = (T["Cs"] * (1 + 0.1 * g.standard_normal(T["Cs"].shape))).astype(np.float32)
    G = (T["G"] + 0.1 * g.standard_normal(T["G"].shape)).astype(np.float32)
    x = wl.mnist_like(5, min(d, 784), seed=2)
    phi = mck.features(plan, torch.from_numpy(x).to(dev), torch.from_numpy(Cs).to(dev),
                       torch.from_numpy(G).to(dev)).cpu().numpy()
    T2 = dict(T, Cs=Cs.astype(np.float64), G=G.astype(np.float64))
    assert _max_err(phi, ff.features(x.astype(np.float64), T2)) <= TOL


@pytest.mark.parametrize("d", [64, 256, 512])
def test_matern(mck, dev, d):
    plan = mck.Plan(d, 2, "matern", 1.0, 1398239763, matern_t=40)
    x = wl.mnist_like(6, min(d, 784), seed=4)
    phi = mck.features(plan, torch.from_numpy(x).to(dev)).cpu().numpy()
    ref = ff.features(x.astype(np.float64), _oracle_tables(plan))
    assert _max_err(phi, ref) <= TOL


@pytest.mark.parametrize("d,E,n", [(8, 3, 5), (64, 3, 7), (1024, 3, 9), (4096, 2, 3)])
def test_laplace(mck, dev, d, E, n):
    """Laplacian calibration through the same kernels. Its radii are heavy
    tailed (chi_d over |N(0,1)|), so a few phases are far larger than the
    RBF's: the bar adds, per phase, float32's resolution of z and the
    rounding of the transform, 2^-24 (|z_k| + 4 log2(d) Cs_k max_j |h_j|),
    with the oracle's own Cs rounded to float32, the precision the library
    stores its tables in (the table tests hold the library's Cs to within
    one float32 ulp of the oracle). Phases past 2e5, where float32 no longer
    resolves a period to 1e-5 at all, are only checked to be bounded."""
    plan = mck.Plan(d, E, "laplace", 3.0, 2024 + d)
    x = wl.mnist_like(n, min(d, 784), seed=d)
    phi = mck.features(plan, torch.from_numpy(x).to(dev)).cpu().numpy().astype(np.float64)
    T = _oracle_tables(plan)
    T["Cs"] = T["Cs"].astype(np.float32).astype(np.float64)
    z = ff.phases(x.astype(np.float64), T)                      # (n, E, d)
    Cs = T["Cs"][None]
    hmax = np.abs(z / Cs).max(axis=2, keepdims=True)
    tol = TOL + 2.0 ** -24 * (np.abs(z) + 4 * max(np.log2(d), 1) * Cs * hmax)
    big = np.abs(z) > 2e5
    tol = np.where(big, 2.0, tol)
    tol = np.concatenate([tol, tol], axis=2).reshape(n, -1)
    ref = ff.features(x.astype(np.float64), T)
    assert np.all(np.abs(phi - ref) <= tol), float((np.abs(phi - ref) - tol).max())
    assert np.all(np.abs(phi) <= 1.0 + 1e-6)
    plan.close()


def test_features_host_pageable_and_large_d(mck, dev):
    """mck_features_host with pageable (not pinned) host arrays, and at
    d = 2^16 where each chunk runs the multi-pass form: equal to the device
    call; a device array is refused."""
    for d, E, n, chunk in ((1024, 2, 45, 16), (1 << 16, 1, 5, 2)):
        plan = mck.Plan(d, E, "rbf", 3.0, 8)
        x = torch.from_numpy(wl.mnist_like(n, 784, seed=n))  # pageable
        out = torch.full((n, plan.num_features), float("nan"))
        mck.features_host(plan, x, out=out, chunk_rows=chunk, streams=3)
        torch.cuda.synchronize()
        assert torch.equal(out, mck.features(plan, x.to(dev)).cpu())
        plan.close()
    plan = mck.Plan(256, 1, "rbf", 1.0, 1)
    pipe = mck.HostPipeline(plan, 200, 8, 2)
    with pytest.raises(mck.MckError, match="device memory"):
        pipe.run(torch.zeros((4, 200), device=dev), torch.zeros((4, plan.num_features)))
    pipe.close()
    plan.close()


@pytest.mark.parametrize("n,chunk,streams", [(1000, 128, 3), (37, 64, 4), (300, 300, 2)])
def test_features_host_pipeline(mck, dev, n, chunk, streams):
    """Host-buffer path: chunks over several streams, copies overlapping the
    kernels; the result equals the device call's bit for bit."""
    plan = mck.Plan(1024, 3, "rbf", 3.0, 5)
    x = torch.from_numpy(wl.mnist_like(n, 784, seed=n)).pin_memory()
    got = mck.features_host(plan, x, chunk_rows=chunk, streams=streams)
    torch.cuda.synchronize()
    ref = mck.features(plan, x.to(dev)).cpu()
    assert torch.equal(got, ref)
    out = torch.full((n, plan.num_features), float("nan")).pin_memory()
    mck.features_host(plan, x, out=out, chunk_rows=chunk, streams=streams)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # a pipeline made once and reused for two batches back to back
    pipe = mck.HostPipeline(plan, 784, chunk, streams)
    x2 = torch.from_numpy(wl.mnist_like(n, 784, seed=n + 1)).pin_memory()
    o1 = mck.features_host(plan, x, pipeline=pipe)
    o2 = mck.features_host(plan, x2, pipeline=pipe)
    torch.cuda.synchronize()
    assert torch.equal(o1, ref)
    assert torch.equal(o2, mck.features(plan, x2.to(dev)).cpu())
    plan.close()


def test_deterministic(mck, dev):
    plan = mck.Plan(1024, 4, "rbf", 1.0, 42)
    x = torch.from_numpy(wl.mnist_like(100, 784, seed=1)).to(dev)
    a = mck.features(plan, x)
    b = mck.features(plan, x)
    assert torch.equal(a, b)


def _sampled_rows_check(mck, dev, N, E, sigma, kernel="rbf"):
    d = 1024
    plan = mck.Plan(d, E, kernel, sigma, 42)
    x = wl.mnist_like(N, 784, seed=42)
    phi = mck.features(plan, torch.from_numpy(x).to(dev))
    rows = np.unique(np.concatenate([[0, 1, 7, 8, N // 2, N - 2, N - 1],
                                     np.random.default_rng(0).integers(0, N, 25)]))
    got = phi[torch.from_numpy(rows).to(dev)].cpu().numpy()
    del phi
    ref = ff.features(x[rows].astype(np.float64), _oracle_tables(plan))
    assert _max_err(got, ref) <= TOL


def test_config1_full_size_sampled(mck, dev):
    # N=60000, E=8, sigma=3, RBF: 3.9 GB of features, checked on sampled rows.
    _sampled_rows_check(mck, dev, 60000, 8, 3.0)


def test_headline_full_size_sampled(mck, dev):
    # N=60000, d=1024, E=16, sigma=3: 7.9 GB of features, checked on sampled rows.
    _sampled_rows_check(mck, dev, 60000, 16, 3.0)
    torch.cuda.empty_cache()
