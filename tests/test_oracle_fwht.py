"""Pins the oracle's Hadamard recursion (Sec. "Fast Walsh Hadamard")."""

import numpy as np
import pytest
import scipy.linalg

from oracle import fastfood as ff


@pytest.mark.parametrize("d", [1, 2, 4, 8, 16, 32, 64])
def test_sylvester_matches_library_and_closed_form(d):
    H = ff.sylvester(d)
    np.testing.assert_array_equal(H, scipy.linalg.hadamard(d))
    i, j = np.meshgrid(np.arange(d), np.arange(d), indexing="ij")
    parity = np.vectorize(lambda a: bin(a).count("1") & 1)(i & j)
    np.testing.assert_array_equal(H, np.where(parity, -1.0, 1.0))


@pytest.mark.parametrize("d", [1, 2, 4, 8, 16, 32, 64])
def test_fwht_brute_force(d):
    rng = np.random.default_rng(d)
    x = rng.standard_normal((5, d))
    np.testing.assert_allclose(ff.fwht(x), x @ scipy.linalg.hadamard(d).T, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d", [2, 128, 4096])
def test_fwht_invariants(d):
    rng = np.random.default_rng(1000 + d)
    x = rng.standard_normal((3, d))
    y = ff.fwht(x)
    # H H = d I
    np.testing.assert_allclose(ff.fwht(y), d * x, rtol=1e-12, atol=1e-9)
    # ||H x||^2 = d ||x||^2
    np.testing.assert_allclose((y ** 2).sum(1), d * (x ** 2).sum(1), rtol=1e-12)
    # H e_0 = ones, H ones = d e_0
    e0 = np.zeros(d); e0[0] = 1.0
    np.testing.assert_array_equal(ff.fwht(e0), np.ones(d))
    ones_t = ff.fwht(np.ones(d))
    np.testing.assert_array_equal(ones_t, d * e0)
    # linearity
    a, b = 0.37, -2.5
    np.testing.assert_allclose(ff.fwht(a * x[0] + b * x[1]), a * y[0] + b * y[1], atol=1e-9)


def test_fwht_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        ff.fwht(np.zeros(6))
