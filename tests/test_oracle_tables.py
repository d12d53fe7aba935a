"""Pins the oracle's hash-driven tables (Sec. "McKernel": B, Pi, G, C; Sec. "Customizing McKernel")."""

import itertools
import math

import numpy as np
import pytest
import scipy.stats

from oracle import fastfood as ff


def test_B_signs_balanced():
    B = ff.table_B(4096, 8, seed=42)
    assert set(np.unique(B)) == {-1.0, 1.0}
    n_neg = int((B < 0).sum())
    n = B.size
    # binomial(n, 1/2): 6 standard deviations
    assert abs(n_neg - n / 2) < 6 * math.sqrt(n / 4)


@pytest.mark.parametrize("d", [2, 16, 1024])
def test_perm_is_permutation(d):
    P = ff.table_perm(d, 3, seed=7)
    for row in P:
        np.testing.assert_array_equal(np.sort(row), np.arange(d))


def test_fisher_yates_draw_range():
    d = 4096
    j = ff.fisher_yates_draws(d, 0, seed=1)
    i = np.arange(d)
    assert np.all(j[1:] >= 0) and np.all(j[1:] <= i[1:])


def test_fisher_yates_uniform_small():
    # d = 3: all 6 permutations equally likely over independent expansions.
    E = 6000
    P = ff.table_perm(3, E, seed=3)
    counts = {p: 0 for p in itertools.permutations(range(3))}
    for row in P:
        counts[tuple(int(v) for v in row)] += 1
    obs = np.array(list(counts.values()))
    chi2 = ((obs - E / 6) ** 2 / (E / 6)).sum()
    assert scipy.stats.chi2.sf(chi2, df=5) > 1e-4


def test_fisher_yates_in_the_papers_words():
    # Sec. "McKernel", Permutation Pi: pick a random element of L, make it the
    # image of n, move n to where the element was removed, and recurse on n-1.
    d = 8
    j = ff.fisher_yates_draws(d, 2, seed=11)
    remaining = list(range(d))
    image = [None] * d
    for n in range(d - 1, 0, -1):
        pos = int(j[n])
        image[n] = remaining[pos]
        remaining[pos] = remaining[n]
        remaining = remaining[:n]
    image[0] = remaining[0]
    np.testing.assert_array_equal(ff.table_perm(d, 3, seed=11)[2], image)


def test_G_is_standard_normal():
    G = ff.table_G(4096, 4, seed=5).ravel()
    assert scipy.stats.kstest(G, "norm").pvalue > 1e-4
    assert abs(G.mean()) < 6 / math.sqrt(G.size)
    assert abs(G.var() - 1) < 6 * math.sqrt(2 / G.size)


def test_box_muller_sin_branch_is_normal():
    w = ff._words(np.arange(20000, dtype=np.uint64), 0, 99, 0, 1)
    c, s = ff.box_muller(w[0], w[1])
    assert scipy.stats.kstest(s, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(c, s)[0, 1]) < 6 / math.sqrt(c.size)


@pytest.mark.parametrize("d", [2, 16, 256, 4096])
def test_rbf_radius_is_chi_d(d):
    ks = range(3000)
    r = ff.table_radius(d, 1, ff.RBF, 0, seed=17, ks=ks)[0]
    assert scipy.stats.kstest(r, scipy.stats.chi(d).cdf).pvalue > 1e-4


@pytest.mark.parametrize("d", [4, 64])
def test_laplace_radius_is_spherical_cauchy(d):
    # The spherical multivariate Cauchy (the Laplacian kernel's spectral
    # density) is z/|n| with z ~ N(0, I_d), n ~ N(0, 1) independent, so
    # r^2/d = (chi2_d/d)/(chi2_1/1) ~ F(d, 1); r > 0 always.
    r = ff.table_radius(d, 1, ff.LAPLACE, 0, seed=19, ks=range(3000))[0]
    assert np.all(r > 0)
    assert scipy.stats.kstest(r ** 2 / d, scipy.stats.f(d, 1).cdf).pvalue > 1e-4
    # the divisor is drawn independently of the chi_d radius of the same k
    q = r / ff.table_radius(d, 1, ff.RBF, 0, seed=19, ks=range(3000))[0]
    assert scipy.stats.kstest(1.0 / q, scipy.stats.halfnorm.cdf).pvalue > 1e-4


def test_matern_single_sample_is_ball_radius():
    # t = 1: ||u_1|| = U^{1/d}, so ||u_1||^d ~ U(0,1) (Sec. "Customizing McKernel": P(R <= r) = r^n).
    d = 8
    r = ff.table_radius(d, 1, ff.MATERN, 1, seed=21, ks=range(3000))[0]
    assert np.all(r <= 1.0)
    assert scipy.stats.kstest(r ** d, "uniform").pvalue > 1e-4


def test_matern_sum_second_moment():
    # u_j i.i.d. uniform in the unit d-ball: E||u||^2 = d/(d+2), E<u_i,u_j> = 0,
    # so E||sum_j u_j||^2 = t d/(d+2).
    d, t = 16, 5
    r = ff.table_radius(d, 1, ff.MATERN, t, seed=23, ks=range(4000))[0]
    m = (r ** 2).mean()
    se = (r ** 2).std() / math.sqrt(r.size)
    assert abs(m - t * d / (d + 2)) < 6 * se


def test_matern_sum_is_rotation_invariant_sum():
    # The norm of a sum of t uniform-ball points: compare with an independent
    # numpy-driven sampler of the same distribution (two-sample KS).
    d, t, n = 8, 3, 3000
    r = ff.table_radius(d, 1, ff.MATERN, t, seed=29, ks=range(n))[0]
    g = np.random.default_rng(0)
    X = g.standard_normal((n, t, d))
    U = g.random((n, t)) ** (1.0 / d)
    ref = np.linalg.norm((U[..., None] * X / np.linalg.norm(X, axis=2, keepdims=True)).sum(1), axis=1)
    assert scipy.stats.ks_2samp(r, ref).pvalue > 1e-4


def test_tables_deterministic_in_seed():
    a = ff.plan_tables(64, 2, ff.RBF, 1.0, seed=9)
    b = ff.plan_tables(64, 2, ff.RBF, 1.0, seed=9)
    c = ff.plan_tables(64, 2, ff.RBF, 1.0, seed=10)
    for k in ("B", "perm", "G", "Cs"):
        np.testing.assert_array_equal(a[k], b[k])
    assert not np.array_equal(a["G"], c["G"])
    # expansions differ from each other
    assert not np.array_equal(a["G"][0], a["G"][1])
