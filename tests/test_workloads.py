"""The seeded input recipes (no GPU): shapes, types, determinism and the
value structure each stand-in is meant to have."""

import numpy as np
import scipy.stats

import workloads as wl


def test_mnist_like_structure():
    x = wl.mnist_like(2000, 784, seed=42)
    assert x.shape == (2000, 784) and x.dtype == np.float32
    assert np.array_equal(x, wl.mnist_like(2000, 784, seed=42))
    assert not np.array_equal(x, wl.mnist_like(2000, 784, seed=43))
    nz = x[x != 0]
    # ~20% nonzero, and the nonzero values uniform on [0, 1)
    assert abs(nz.size / x.size - 0.2) < 0.005
    assert nz.min() >= 0 and nz.max() < 1
    assert scipy.stats.kstest(nz[:20000], "uniform").pvalue > 1e-4


def test_gaussian_and_labels():
    g = wl.gaussian(500, 256, seed=7)
    assert g.shape == (500, 256) and g.dtype == np.float32
    assert scipy.stats.kstest(g.ravel()[:50000], "norm").pvalue > 1e-4
    y = wl.labels(5000, 10, seed=3)
    assert y.dtype == np.int32 and y.min() >= 0 and y.max() <= 9
    assert scipy.stats.chisquare(np.bincount(y, minlength=10)).pvalue > 1e-4


def test_logit_weights_and_teacher_labels():
    W, b = wl.logit_weights(10, 4096, seed=1)
    assert W.shape == (10, 4096) and W.dtype == np.float32 and np.all(b == 0)
    assert abs(W.std() - 0.01) < 0.0005
    x = wl.mnist_like(3000, 100, seed=5)
    t = wl.teacher_labels(x, 10, seed=2)
    assert t.dtype == np.int32 and t.shape == (3000,)
    assert len(np.unique(t)) == 10  # every class occurs


def test_uneven_batch_recipe():
    b = wl.uneven_batch(4000, seed=42)
    d, E, k = b["d"], b["E"], b["kernel"]
    assert set(np.unique(np.log2(d).astype(int))) == set(range(6, 15))
    assert E.min() >= 1 and E.max() <= 32 and set(np.unique(k)) == {0, 1}
    assert all(len(v) == di and v.dtype == np.float32 for v, di in zip(b["x"][:50], d[:50]))
    b2 = wl.uneven_batch(4000, seed=42)
    assert np.array_equal(d, b2["d"]) and np.array_equal(b["x"][7], b2["x"][7])
