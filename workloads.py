"""Seeded synthetic inputs for the McKernel feature map.

This module only draws input data; it holds none of the method's arithmetic.
Both the tests (oracle side and CUDA side) and ``bench.py`` take their inputs
from here, so the two sides always see the same numbers. All arrays are
float32 (the CUDA path's input type; the oracle widens them to float64
exactly). Generator: numpy ``Generator(PCG64(seed))``.

Stand-ins for the paper's data (Sec. "Empirical Analysis and Experiments"):
MNIST and FASHION-MNIST images (784 = 28 x 28 pixels, padded to d = 1024) are
replaced by rows with ~80% exact zeros and the other entries uniform in [0, 1),
which is the value structure of a normalised MNIST digit. The datasets
themselves are not used.
"""

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def mnist_like(n, in_dim=784, seed=42, p_nonzero=0.2):
    """(n, in_dim) float32: each entry 0 with prob 1-p_nonzero, else U[0,1)."""
    g = _rng(seed)
    vals = g.random((n, in_dim), dtype=np.float32)
    keep = g.random((n, in_dim), dtype=np.float32) < p_nonzero
    return np.where(keep, vals, np.float32(0.0)).astype(np.float32)


def gaussian(n, d, seed=42):
    """(n, d) float32 with i.i.d. N(0, 1) entries."""
    return _rng(seed).standard_normal((n, d), dtype=np.float32)


def labels(n, num_classes=10, seed=42):
    """(n,) int32 labels uniform on 0..num_classes-1."""
    return _rng(seed).integers(0, num_classes, size=n, dtype=np.int32)


def teacher_labels(x, num_classes=10, seed=42):
    """Labels a classifier can learn: argmax of a fixed random linear map of
    the centred inputs (entries of the map N(0,1)), as int32."""
    g = _rng(seed)
    V = g.standard_normal((x.shape[1], num_classes))
    return np.argmax((x - x.mean(axis=0)) @ V, axis=1).astype(np.int32)


def logit_weights(num_classes, num_features, seed=42, std=0.01):
    """W (C, F) float32 ~ N(0, std^2) and b = 0 (C,) float32."""
    W = (_rng(seed).standard_normal((num_classes, num_features), dtype=np.float32)
         * np.float32(std)).astype(np.float32)
    return W, np.zeros(num_classes, dtype=np.float32)


def uneven_batch(count=10000, seed=42, log2_d=(6, 14), max_E=32):
    """The serving-style mix: per vector log2(d) ~ U{6..14}, E ~ U{1..32},
    kernel ~ Bernoulli(1/2) (0 = RBF, 1 = Matern), entries N(0,1).

    Returns dict with int arrays ``d``, ``E``, ``kernel`` and a list ``x`` of
    float32 vectors of length d_i.
    """
    g = _rng(seed)
    m = g.integers(log2_d[0], log2_d[1] + 1, size=count)
    d = (1 << m).astype(np.int64)
    E = g.integers(1, max_E + 1, size=count).astype(np.int64)
    kernel = g.integers(0, 2, size=count).astype(np.int64)
    x = [g.standard_normal(int(di), dtype=np.float32) for di in d]
    return {"d": d, "E": E, "kernel": kernel, "x": x}
