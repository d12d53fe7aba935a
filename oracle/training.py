"""softmax(W phi + b), cross-entropy and gradients, numpy float64 (test infrastructure only).

Only tests, the smoke check and the benchmark's CPU-baseline leg use this
module; the CUDA library never does.

Sec. "Empirical Analysis and Experiments": SGD finds W and b in
softmax(W phi(Z-hat x-hat) + b). The paper's loss (Eq. etn:loss) is the
logistic loss log(1 + exp(-y f)); with C classes its multi-class form is the
softmax cross-entropy -log softmax(l)_y, which equals the logistic loss when
C = 2 (tests check that reduction). Sec. "Empirical Analysis" also proposes
learning the calibration C and G by backpropagation, and learning B (which
it likens to attention), so gradients are given with respect to x, Cs
(= C/(sigma sqrt d)), G, W, b and B. For B the map is read with B as a real
diagonal (u0 = B x-hat, linear in B); a trainer that keeps B in {+1, -1}
passes this gradient through the sign (straight-through).

Gradients follow the chain rule through each stage of
z = Cs H G Pi H B x-hat using H^T = H and Pi^T = Pi^{-1}:
  dz  = -sin z * dphi_cos + cos z * dphi_sin
  dCs = sum_n h * dz,   dh = Cs * dz,   dw = H dh
  dG  = sum_n v * dw,   dv = G * dw,    du[perm[k]] = dv[k],   du0 = H du
  dx  = sum_e (B * du0)[:in_dim]
  dB  = sum_n x-hat * du0
Pinned by central finite differences of ``loss`` (tests/test_oracle_training.py).
"""

import numpy as np

from . import fastfood as ff


def logits(phi, W, b):
    """l = phi W^T + b; phi (N, F), W (C, F), b (C,)."""
    return phi @ W.T + b


def softmax_xent(l, y):
    """Mean cross-entropy of softmax(l) against integer labels y, and dl."""
    l = np.asarray(l, dtype=np.float64)
    m = l.max(axis=1, keepdims=True)
    lse = m[:, 0] + np.log(np.exp(l - m).sum(axis=1))
    N = l.shape[0]
    loss = float(np.mean(lse - l[np.arange(N), y]))
    p = np.exp(l - lse[:, None])
    dl = p.copy()
    dl[np.arange(N), y] -= 1.0
    return loss, dl / N


def loss(x, T, W, b, y):
    phi = ff.features(x, T)
    return softmax_xent(logits(phi, W, b), y)[0]


def features_backward(x, T, dphi, with_dB=False):
    """Gradients of sum(phi * dphi) w.r.t. x, Cs and G (chain rule, see header);
    with ``with_dB`` also w.r.t. the diagonal B, as a fourth result."""
    B, perm, G, Cs = T["B"], T["perm"], T["G"], T["Cs"]
    E, d = B.shape
    N, in_dim = x.shape
    dphi = dphi.reshape(N, E, 2, d)
    dx_hat = np.zeros((N, d))
    dCs = np.zeros((E, d))
    dG = np.zeros((E, d))
    dB = np.zeros((E, d))
    xh = ff.pad(x, d)
    for e in range(E):
        s = ff.stages(x, B[e], perm[e], G[e], Cs[e])
        z = s["z"]
        dz = -np.sin(z) * dphi[:, e, 0, :] + np.cos(z) * dphi[:, e, 1, :]
        dCs[e] = (s["h"] * dz).sum(axis=0)
        dh = Cs[e] * dz
        dw = ff.fwht(dh)
        dG[e] = (s["v"] * dw).sum(axis=0)
        dv = G[e] * dw
        du = np.zeros_like(dv)
        du[:, perm[e]] = dv
        du0 = ff.fwht(du)
        dx_hat += B[e] * du0
        dB[e] = (xh * du0).sum(axis=0)
    if with_dB:
        return dx_hat[:, :in_dim], dCs, dG, dB
    return dx_hat[:, :in_dim], dCs, dG


def train_grads(x, T, W, b, y):
    """Loss and every gradient of the softmax cross-entropy of W phi + b."""
    phi = ff.features(x, T)
    l = logits(phi, W, b)
    L, dl = softmax_xent(l, y)
    dW = dl.T @ phi
    db = dl.sum(axis=0)
    dphi = dl @ W
    dx, dCs, dG, dB = features_backward(x, T, dphi, with_dB=True)
    return {"loss": L, "logits": l, "dlogits": dl, "dW": dW, "db": db,
            "dx": dx, "dCs": dCs, "dG": dG, "dB": dB}


def finite_difference(f, a, idx, h=1e-6):
    """Central difference (f(a + h e_i) - f(a - h e_i)) / 2h for each flat index i."""
    out = []
    flat = a.reshape(-1)
    for i in idx:
        old = flat[i]
        flat[i] = old + h
        fp = f()
        flat[i] = old - h
        fm = f()
        flat[i] = old
        out.append((fp - fm) / (2.0 * h))
    return np.array(out)
