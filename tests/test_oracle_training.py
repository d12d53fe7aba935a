"""Pins the oracle's logits, loss and gradients (Sec. "TIKHONOV", Sec. "Empirical Analysis")."""

import numpy as np
import pytest
import scipy.special

from oracle import fastfood as ff
from oracle import training as tr


def test_two_class_softmax_is_logistic_loss():
    # Eq. etn:loss: l(y, f) = log(1 + exp(-y f)); softmax over 2 classes with
    # f = l_1 - l_0 and y = +1 for class 1, -1 for class 0.
    g = np.random.default_rng(0)
    l = g.standard_normal((50, 2)) * 3
    lab = g.integers(0, 2, 50)
    loss, _ = tr.softmax_xent(l, lab)
    y = 2.0 * lab - 1.0
    f = l[:, 1] - l[:, 0]
    assert abs(loss - np.mean(np.log1p(np.exp(-y * f)))) < 1e-12


def test_softmax_xent_against_logsumexp():
    g = np.random.default_rng(1)
    l = g.standard_normal((20, 10)) * 5
    lab = g.integers(0, 10, 20)
    loss, dl = tr.softmax_xent(l, lab)
    ref = np.mean(scipy.special.logsumexp(l, axis=1) - l[np.arange(20), lab])
    assert abs(loss - ref) < 1e-12
    np.testing.assert_allclose(dl.sum(axis=1), 0.0, atol=1e-15)


@pytest.fixture(scope="module")
def problem():
    d, E, C, N, in_dim = 64, 2, 3, 4, 50
    T = ff.plan_tables(d, E, ff.RBF, 1.0, seed=5)
    g = np.random.default_rng(7)
    x = g.random((N, in_dim))
    W = g.standard_normal((C, 2 * E * d)) * 0.1
    b = g.standard_normal(C) * 0.1
    y = g.integers(0, C, N)
    return T, x, W, b, y


def _check(analytic, numeric):
    err = np.abs(analytic - numeric).max() / max(np.abs(numeric).max(), 1e-12)
    assert err < 1e-6, err


def test_grads_against_central_differences(problem):
    T, x, W, b, y = problem
    T = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in T.items()}
    x, W, b = x.copy(), W.copy(), b.copy()
    g = tr.train_grads(x, T, W, b, y)
    f = lambda: tr.loss(x, T, W, b, y)
    rng = np.random.default_rng(3)
    idx_w = rng.choice(W.size, 40, replace=False)
    idx_x = rng.choice(x.size, 40, replace=False)
    _check(g["db"], tr.finite_difference(f, b, range(b.size)))
    _check(g["dW"].ravel()[idx_w], tr.finite_difference(f, W, idx_w))
    _check(g["dCs"].ravel(), tr.finite_difference(f, T["Cs"], range(T["Cs"].size)))
    _check(g["dG"].ravel(), tr.finite_difference(f, T["G"], range(T["G"].size)))
    _check(g["dx"].ravel()[idx_x], tr.finite_difference(f, x, idx_x))
    # B as a real diagonal (u0 = B x-hat): the loss is smooth in it
    T["B"] = T["B"].astype(np.float64)
    _check(g["dB"].ravel(), tr.finite_difference(f, T["B"], range(T["B"].size)))


def test_sign_gradient_zero_past_input(problem):
    # Coordinates k >= in_dim of x-hat are zero padding: B has no effect there.
    T, x, W, b, y = problem
    g = tr.train_grads(x, T, W, b, y)
    assert np.all(g["dB"][:, x.shape[1]:] == 0.0)
    assert np.abs(g["dB"][:, : x.shape[1]]).max() > 0


def test_features_backward_is_adjoint(problem):
    # <dphi, J v> = <J^T dphi, v> for a random direction v in x: the backward is
    # the exact transpose of the forward's Jacobian.
    T, x, W, b, y = problem
    g = np.random.default_rng(11)
    dphi = g.standard_normal((x.shape[0], 2 * 2 * 64))
    v = g.standard_normal(x.shape)
    h = 1e-6
    jv = (ff.features(x + h * v, T) - ff.features(x - h * v, T)) / (2 * h)
    dx, _, _ = tr.features_backward(x, T, dphi)
    assert abs((dphi * jv).sum() - (dx * v).sum()) < 1e-6 * abs((dx * v).sum()) + 1e-9
