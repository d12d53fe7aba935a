"""The plain FP32 CPU baseline (cpu_baseline/) against the FP64 oracle (CPU only).

The baseline is what the benchmark times as the multi-core CPU version of
the method, so its features must be the method's: within 1e-5 of the oracle
at MNIST-shaped phases, the same for any thread count, and written to row
i % out_rows of a wrap-around output buffer.
"""

import numpy as np
import pytest

import cpu_baseline as cb
import workloads as wl
from oracle import fastfood as ff


def _tables32(d, E, kernel=ff.RBF, sigma=3.0, seed=42):
    T = ff.plan_tables(d, E, kernel, sigma, seed=seed)
    return T, (T["B"].astype(np.float32), T["perm"].astype(np.uint32),
               T["G"].astype(np.float32), T["Cs"].astype(np.float32))


@pytest.mark.parametrize("d,E,in_dim", [(2, 3, 2), (8, 2, 5), (64, 3, 64),
                                        (1024, 2, 784), (4096, 1, 3000)])
def test_matches_oracle(d, E, in_dim):
    x = wl.mnist_like(6, in_dim, seed=d)
    T, tabs = _tables32(d, E)
    got = cb.features(x, *tabs, threads=2)
    # the oracle on the float32-rounded tables the baseline is given
    T32 = dict(T, G=tabs[2].astype(np.float64), Cs=tabs[3].astype(np.float64))
    ref = ff.features(x.astype(np.float64), T32)
    assert got.shape == ref.shape
    assert float(np.abs(got - ref).max()) <= 1e-5


def test_thread_count_does_not_change_results():
    x = wl.mnist_like(37, 784, seed=3)
    _, tabs = _tables32(1024, 2)
    a = cb.features(x, *tabs, threads=1)
    b = cb.features(x, *tabs, threads=5)
    assert np.array_equal(a, b)


def test_wrap_around_output_rows():
    x = wl.mnist_like(5, 60, seed=4)
    _, tabs = _tables32(64, 2)
    full = cb.features(x, *tabs, threads=1)
    out = np.zeros((2, full.shape[1]), np.float32)
    cb.features(x, *tabs, threads=1, out=out)
    assert np.array_equal(out[0], full[4]) and np.array_equal(out[1], full[3])


def test_bad_arguments_are_refused():
    lib = cb.load()
    assert lib.ff32_features(None, 1, 3, 3, 6, 1, None, None, None, None, None, 1, 1) == -1  # d not 2^k
    assert lib.ff32_features(None, 0, 3, 3, 8, 1, None, None, None, None, None, 1, 1) == 0   # n = 0
    assert lib.ff32_features(None, 2, 9, 9, 8, 1, None, None, None, None, None, 1, 1) == -1  # in_dim > d
