"""Pins the oracle's map Z-hat (Eq. etn:mckernel) and features (Eq. etn:mcfeatures)."""

import math

import numpy as np
import pytest
import scipy.linalg
import scipy.special

from oracle import fastfood as ff


def _explicit_zhat(T, e, sigma):
    """Z-hat_e from dense matrices: (1/(sigma sqrt d)) C H G Pi H B."""
    d = T["B"].shape[1]
    H = scipy.linalg.hadamard(d).astype(np.float64)
    P = np.zeros((d, d))
    P[np.arange(d), T["perm"][e]] = 1.0          # (P v)_k = v_{perm[k]}
    M = np.diag(T["C"][e]) @ H @ np.diag(T["G"][e]) @ P @ H @ np.diag(T["B"][e])
    return M / (sigma * math.sqrt(d))


@pytest.mark.parametrize("d,kernel", [(2, ff.RBF), (16, ff.RBF), (64, ff.RBF), (32, ff.MATERN)])
def test_zhat_matches_dense_product(d, kernel):
    sigma = 1.7
    T = ff.plan_tables(d, 2, kernel, sigma, t=5, seed=3)
    for e in range(2):
        np.testing.assert_allclose(ff.zhat_matrix(T, e), _explicit_zhat(T, e, sigma), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [4, 32, 64])
def test_zhat_row_norms(d):
    # Row k of H G Pi H B has norm sqrt(d) ||G||, so row k of Z-hat has norm
    # C[k] ||G|| / sigma = r_k / sigma: the calibration sets each row's length.
    sigma = 0.8
    T = ff.plan_tables(d, 3, ff.RBF, sigma, seed=5)
    for e in range(3):
        norms = np.linalg.norm(ff.zhat_matrix(T, e), axis=1)
        np.testing.assert_allclose(norms, T["r"][e] / sigma, rtol=1e-12)


def _pair(d, dist, seed):
    g = np.random.default_rng(seed)
    x = g.standard_normal(d) * 0.3
    u = g.standard_normal(d)
    return x, x + dist * u / np.linalg.norm(u)


@pytest.mark.parametrize("s", [0.25, 0.5, 1.0, 2.0])
def test_rbf_kernel_approximation(s):
    # phi(x).phi(y) / (E d) = mean_k cos(w_k . (x - y)) -> exp(-||x-y||^2 / (2 sigma^2))  (Eq. etn:rbf)
    d, E, sigma = 64, 64, 1.5
    T = ff.plan_tables(d, E, ff.RBF, sigma, seed=31)
    x, y = _pair(d, s * sigma, seed=int(s * 100))
    phi = ff.features(np.stack([x, y]), T)
    est = phi[0] @ phi[1] / (E * d)
    assert abs(est - math.exp(-s * s / 2)) < 5 / math.sqrt(E * d)
    # A dropped sqrt(d) or ||G|| normalisation would move the estimate far off:
    assert abs(phi[0] @ phi[0] / (E * d) - 1.0) < 1e-12


@pytest.mark.parametrize("s", [0.25, 0.5, 1.0])
def test_laplace_kernel_approximation(s):
    # |w_k| = r_k / sigma with r_k ~ chi_d/|N(0,1)| and a (nearly) uniform
    # direction: E cos(w . Delta) = exp(-||Delta|| / sigma), the Laplacian kernel.
    d, E, sigma = 64, 64, 1.5
    T = ff.plan_tables(d, E, ff.LAPLACE, sigma, seed=33)
    x, y = _pair(d, s * sigma, seed=int(s * 100) + 1)
    phi = ff.features(np.stack([x, y]), T)
    est = phi[0] @ phi[1] / (E * d)
    assert abs(est - math.exp(-s)) < 5 / math.sqrt(E * d)
    # at these distances the Gaussian's value lies outside the bar
    assert abs(math.exp(-s) - math.exp(-s * s / 2)) > 5 / math.sqrt(E * d)


def _ball_charfn(d, s):
    """E exp(i w.u) for u uniform in the unit d-ball, |w| = s: Gamma(d/2+1) (2/s)^{d/2} J_{d/2}(s)."""
    nu = d / 2.0
    return math.exp(math.lgamma(nu + 1) + nu * math.log(2.0 / s)) * scipy.special.jv(nu, s)


@pytest.mark.parametrize("s", [0.5, 1.0, 2.0])
def test_matern_kernel_approximation(s):
    # w = (sum of t uniform-ball points)/sigma, so E cos(w.Delta) = charfn(|Delta|/sigma)^t.
    d, E, t, sigma = 16, 48, 5, 0.7
    T = ff.plan_tables(d, E, ff.MATERN, sigma, t=t, seed=37)
    x, y = _pair(d, s * sigma, seed=int(s * 10) + 1)
    phi = ff.features(np.stack([x, y]), T)
    est = phi[0] @ phi[1] / (E * d)
    assert abs(est - _ball_charfn(d, s) ** t) < 5 / math.sqrt(E * d)


def test_ball_charfn_small_argument():
    # Sanity of the closed form itself: charfn(s) ~ 1 - s^2/(2(d+2)) for small s.
    for d in (2, 8, 64):
        s = 1e-3
        assert abs(_ball_charfn(d, s) - (1 - s * s / (2 * (d + 2)))) < 1e-10


def test_padding_and_linearity():
    d = 64
    T = ff.plan_tables(d, 2, ff.RBF, 1.0, seed=41)
    g = np.random.default_rng(1)
    x = g.standard_normal((3, 50))
    np.testing.assert_array_equal(ff.features(x, T), ff.features(ff.pad(x, d), T))
    a, b = 0.3, -1.7
    za = ff.phases(a * x[:1] + b * x[1:2], T)
    np.testing.assert_allclose(za, a * ff.phases(x[:1], T) + b * ff.phases(x[1:2], T), atol=1e-12)


def test_feature_layout_and_parameter_count():
    # Output per sample: E blocks of [cos (d) | sin (d)], 2 d E values; the
    # paper's parameter count for C classes is C (2 [S]_2 E + 1) (Sec. "Empirical Analysis").
    d, E, C = 16, 3, 10
    T = ff.plan_tables(d, E, ff.RBF, 1.0, seed=43)
    x = np.random.default_rng(2).standard_normal((2, 10))
    z = ff.phases(x, T)
    phi = ff.features(x, T)
    assert phi.shape == (2, 2 * d * E)
    for e in range(E):
        np.testing.assert_array_equal(phi[:, 2 * d * e: 2 * d * e + d], np.cos(z[:, e]))
        np.testing.assert_array_equal(phi[:, 2 * d * e + d: 2 * d * (e + 1)], np.sin(z[:, e]))
    assert C * (phi.shape[1] + 1) == 10 * (2 * 16 * 3 + 1)
    assert 10 * (2 * 1024 * 16 + 1) == 327690
