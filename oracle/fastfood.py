"""Fastfood / McKernel map in plain numpy float64 (test infrastructure only).

Only tests, the smoke check and the benchmark's CPU-baseline leg use this
module; the CUDA library never does, and this module imports nothing from it.

Notation follows the paper (arXiv 1702.08159):
  d      padded input dimension, a power of two (the paper's ``n`` in
         Eq. etn:mckernel and ``[x]_2`` in Sec. "Empirical Analysis").
  E      number of kernel expansions (i.i.d. copies of Z-hat, Sec. "McKernel").
  B      diagonal of random signs            (Sec. "McKernel", "Binary B").
  H      unnormalised Sylvester Hadamard     (Sec. "Fast Walsh Hadamard").
  Pi     random permutation, Fisher-Yates    (Sec. "McKernel", "Permutation Pi").
  G      diagonal Gaussian via Box-Muller    (Sec. "McKernel", "Gaussian G").
  C      calibration diagonal                (Sec. "McKernel", "Calibration C";
         Sec. "Customizing McKernel" for the Matern kernel). Fastfood (Le et
         al.) calls it S.
  Z-hat  = (1/(sigma sqrt d)) C H G Pi H B   (Eq. etn:mckernel).
  phi    = [cos(Z-hat x), sin(Z-hat x)] per expansion (Eq. etn:mcfeatures).

Random draws come from Philox4x32-10 (``oracle.philox``) with the counter
layout (c0, c1, c2, c3) = (index, expansion e, tag, sub-draw) and key = the
64-bit seed split into two words. Tags:
  1 B sign, 2 Fisher-Yates draw, 3 G, 4 RBF radius (Marsaglia-Tsang trial),
  5 Matern ball coordinates (c2 = 5 + 16*k), 6 Matern ball radius,
  7 the normal divisor of the Laplacian radius.

Readings of points the paper leaves open:
  * B[k] = -1 when bit 0 of word 0 is set, else +1.
  * Fisher-Yates draws j = floor(w0 * (i+1) / 2**32) for i = d-1 .. 1 and swaps
    L[i], L[j]; (Pi v)_k = v_{pi(k)} (a gather).
  * Box-Muller uses u1 = (w0+1)/2**32 in (0,1], u2 = w1/2**32 in [0,1); G uses
    the cosine branch only, one normal per counter.
  * RBF calibration (the paper only says it depends on the kernel): as in
    Fastfood, C[k] = r_k / ||G_e||_2 with r_k ~ chi_d, so each row of Z-hat has
    norm r_k / sigma, i.e. the rows are N(0, I/sigma^2) in distribution. r_k^2
    is drawn as 2*Gamma(d/2, 1) by Marsaglia & Tsang's (2000) exact rejection
    method.
  * Matern calibration, the paper's algorithm literally: r_k = || sum_{j=1..t}
    u_j || with u_j = U_j^{1/d} X_j/||X_j||, X_j ~ N(0, I_d), U_j ~ U(0,1];
    again C[k] = r_k / ||G_e||_2.
  * Laplacian calibration, one more "radial spectral distribution" (Sec.
    "McKernel", item C): the kernel exp(-||x - y|| / sigma) has the spherical
    multivariate Cauchy as spectral density, whose radius is chi_d / |N(0,1)|;
    r_k = (the RBF radius) / max(|n_k|, 2**-32) with n_k the Box-Muller
    (cosine) normal of counter (k, e, 7, 0); again C[k] = r_k / ||G_e||_2.
  * The 1/(sigma sqrt d) factor is applied with C: Cs = C / (sigma sqrt d).
  * phi = [cos | sin] per expansion block, no 1/sqrt(E d) normalisation.
  * x-hat = x followed by zeros (padding at the end).

Parity: every function here is pinned by tests/test_oracle_*.py (Sylvester
brute force, Hadamard invariants, Random123 answers, distribution tests,
closed-form RBF / Matern kernels, row norms of Z-hat).
"""

import math

import numpy as np

from .philox import philox4x32_10, seed_key

TAG_B = 1
TAG_PERM = 2
TAG_G = 3
TAG_RBF = 4
TAG_BALL = 5
TAG_BALL_RADIUS = 6
TAG_LAPLACE = 7

RBF = 0
MATERN = 1
LAPLACE = 2

TWO_M32 = 2.0 ** -32


# ----------------------------------------------------------------------------
# Hadamard (Sec. "Fast Walsh Hadamard")
# ----------------------------------------------------------------------------

def sylvester(d):
    """Explicit H with H_0 = [1] and H_n = [[H_{n-1}, H_{n-1}], [H_{n-1}, -H_{n-1}]]."""
    if d < 1 or d & (d - 1):
        raise ValueError("d must be a power of two")
    h = np.ones((1, 1))
    while h.shape[0] < d:
        h = np.block([[h, h], [h, -h]])
    return h


def fwht(c):
    """H c along the last axis by the paper's divide and conquer.

    With c = (c0, c1) split in halves, H_n c = [H_{n-1} c0 + H_{n-1} c1,
    H_{n-1} c0 - H_{n-1} c1]; both halves are transformed by one recursive
    call on a (..., 2, d/2) view. Unnormalised; T(n) = 2T(n/2) + O(n).
    """
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[-1]
    if n & (n - 1) or n == 0:
        raise ValueError("length must be a power of two")
    if n == 1:
        return c.copy()
    h = n // 2
    halves = fwht(c.reshape(c.shape[:-1] + (2, h)))
    c0 = halves[..., 0, :]
    c1 = halves[..., 1, :]
    return np.concatenate([c0 + c1, c0 - c1], axis=-1)


# ----------------------------------------------------------------------------
# Hash-driven tables (Sec. "McKernel", items B, Pi, G, C)
# ----------------------------------------------------------------------------

def _words(idx, e, tag, sub, seed):
    k0, k1 = seed_key(seed)
    return philox4x32_10(idx, e, tag, sub, k0, k1)


def _unit_open0(w):
    """(w + 1) / 2**32, in (0, 1]."""
    return (w.astype(np.float64) + 1.0) * TWO_M32


def _unit_closed0(w):
    """w / 2**32, in [0, 1)."""
    return w.astype(np.float64) * TWO_M32


def box_muller(w0, w1):
    """Box & Muller (1958): R = sqrt(-2 ln u1), angle 2 pi u2; returns (R cos, R sin)."""
    r = np.sqrt(-2.0 * np.log(_unit_open0(w0)))
    a = 2.0 * np.pi * _unit_closed0(w1)
    return r * np.cos(a), r * np.sin(a)


def table_B(d, E, seed):
    """Signs B_e[k] in {+1, -1}, shape (E, d)."""
    k = np.arange(d, dtype=np.uint64)[None, :]
    e = np.arange(E, dtype=np.uint64)[:, None]
    w0, _, _, _ = _words(k, e, TAG_B, 0, seed)
    return np.where(w0 & 1, -1.0, 1.0)


def fisher_yates_draws(d, e, seed):
    """The index drawn at each step i = 1..d-1: j_i uniform on {0..i}."""
    i = np.arange(d, dtype=np.uint64)
    w0, _, _, _ = _words(i, e, TAG_PERM, 0, seed)
    return ((w0.astype(np.uint64) * (i + np.uint64(1))) >> np.uint64(32)).astype(np.int64)


def table_perm(d, E, seed):
    """pi_e by Durstenfeld's Fisher-Yates on L = [0..d-1], shape (E, d), int64.

    Step i (from d-1 down to 1) picks position j in {0..i}; that element becomes
    the image of i and the element at i moves to position j (a swap).
    """
    out = np.empty((E, d), dtype=np.int64)
    for e in range(E):
        j = fisher_yates_draws(d, e, seed)
        L = list(range(d))
        for i in range(d - 1, 0, -1):
            ji = int(j[i])
            L[i], L[ji] = L[ji], L[i]
        out[e] = L
    return out


def table_G(d, E, seed):
    """G_e[k] ~ N(0,1) by Box-Muller (cosine branch), shape (E, d)."""
    k = np.arange(d, dtype=np.uint64)[None, :]
    e = np.arange(E, dtype=np.uint64)[:, None]
    w0, w1, _, _ = _words(k, e, TAG_G, 0, seed)
    g, _ = box_muller(w0, w1)
    return g


def rbf_radius(d, e, k, seed, max_trials=64):
    """r ~ chi_d: r^2 = 2 Gamma(d/2, 1) by Marsaglia & Tsang (2000).

    a = d/2 >= 1, dd = a - 1/3, c = 1/sqrt(9 dd). Trial j draws a normal g
    (Box-Muller of words 0, 1) and U = (w2 + 1)/2**32 from counter (k, e, 4, j);
    v = (1 + c g)^3 must be positive and the trial is accepted when
    ln U < g^2/2 + dd - dd v + dd ln v. Then r^2 = 2 dd v.
    """
    a = d / 2.0
    dd = a - 1.0 / 3.0
    c = 1.0 / math.sqrt(9.0 * dd)
    for j in range(max_trials):
        w0, w1, w2, _ = _words(np.uint64(k), np.uint64(e), TAG_RBF, j, seed)
        g, _ = box_muller(w0, w1)
        g = float(g)
        u = float(_unit_open0(w2))
        v = 1.0 + c * g
        if v <= 0.0:
            continue
        v = v * v * v
        if math.log(u) < 0.5 * g * g + dd - dd * v + dd * math.log(v):
            return math.sqrt(2.0 * dd * v)
    raise RuntimeError("Marsaglia-Tsang did not accept within max_trials")


def ball_sum_norm(d, e, k, t, seed):
    """|| sum_{j=1..t} u_j || with u_j uniform in the unit d-ball.

    Sec. "Customizing McKernel": X ~ N(0, I_d), Y = X/||X|| is uniform on the
    sphere and U^{1/d} Y is uniform in the ball. Coordinates 2p and 2p+1 of X_j
    are the Box-Muller pair of counter (p, e, 5 + 16 k, j); U_j = (w0+1)/2**32
    of counter (k, e, 6, j).
    """
    p = np.arange(d // 2, dtype=np.uint64)[None, :]
    j = np.arange(1, t + 1, dtype=np.uint64)[:, None]
    w0, w1, _, _ = _words(p, e, TAG_BALL + 16 * k, j, seed)      # (t, d/2)
    xc, xs = box_muller(w0, w1)
    X = np.empty((t, d))
    X[:, 0::2] = xc
    X[:, 1::2] = xs
    u0, _, _, _ = _words(np.uint64(k), np.uint64(e), TAG_BALL_RADIUS, j[:, 0], seed)
    rho = _unit_open0(u0) ** (1.0 / d)                            # (t,)
    u = rho[:, None] * X / np.linalg.norm(X, axis=1, keepdims=True)  # t ball samples
    return float(np.linalg.norm(u.sum(axis=0)))


def laplace_radius(d, e, k, seed):
    """r = chi_d / |N(0,1)|: the radius of the spherical multivariate Cauchy,
    the spectral density of exp(-||x - y||) (a multivariate t with one degree
    of freedom: z / |n| with z ~ N(0, I_d), n ~ N(0, 1) independent). The
    divisor is floored at 2**-32 (a zero draw has probability 2**-32)."""
    w0, w1, _, _ = _words(np.uint64(k), np.uint64(e), TAG_LAPLACE, 0, seed)
    n, _ = box_muller(w0, w1)
    return rbf_radius(d, e, k, seed) / max(abs(float(n)), TWO_M32)


def table_radius(d, E, kernel, t, seed, ks=None):
    """Row norms r_e[k] of the calibration, shape (E, len(ks))."""
    ks = range(d) if ks is None else ks
    out = np.empty((E, len(ks)))
    for e in range(E):
        for i, k in enumerate(ks):
            if kernel == RBF:
                out[e, i] = rbf_radius(d, e, k, seed)
            elif kernel == LAPLACE:
                out[e, i] = laplace_radius(d, e, k, seed)
            else:
                out[e, i] = ball_sum_norm(d, e, k, t, seed)
    return out


def plan_tables(d, E, kernel=RBF, sigma=1.0, t=40, seed=0):
    """All tables of one plan: dict with B, perm, G, C and Cs = C/(sigma sqrt d)."""
    if d < 2 or d & (d - 1):
        raise ValueError("d must be a power of two >= 2")
    B = table_B(d, E, seed)
    perm = table_perm(d, E, seed)
    G = table_G(d, E, seed)
    r = table_radius(d, E, kernel, t, seed)
    C = r / np.linalg.norm(G, axis=1, keepdims=True)
    Cs = C / (sigma * math.sqrt(d))
    return {"B": B, "perm": perm, "G": G, "C": C, "Cs": Cs, "r": r}


# ----------------------------------------------------------------------------
# The map (Eq. etn:mckernel) and the features (Eq. etn:mcfeatures)
# ----------------------------------------------------------------------------

def pad(x, d):
    """x-hat = [x, 0, ..., 0] of length d (Fig. 1 caption; x-hat = [x]_2)."""
    x = np.asarray(x, dtype=np.float64)
    if x.shape[-1] > d:
        raise ValueError("input longer than d")
    out = np.zeros(x.shape[:-1] + (d,))
    out[..., : x.shape[-1]] = x
    return out


def stages(x, B, perm, G, Cs):
    """Every intermediate of z = Cs H G Pi H B x-hat for one expansion.

    x: (N, in_dim); B, perm, G, Cs: (d,). Returns dict with u0 = B x-hat,
    u = H u0, v = Pi u (v_k = u_{perm[k]}), w = G v, h = H w, z = Cs h.
    """
    d = B.shape[-1]
    xh = pad(x, d)
    u0 = B * xh
    u = fwht(u0)
    v = u[..., perm]
    w = G * v
    h = fwht(w)
    z = Cs * h
    return {"u0": u0, "u": u, "v": v, "w": w, "h": h, "z": z}


def phases(x, T):
    """z for every expansion, shape (N, E, d); T is a dict from ``plan_tables``
    (or one with learned ``G`` / ``Cs`` swapped in)."""
    E = T["B"].shape[0]
    return np.stack([stages(x, T["B"][e], T["perm"][e], T["G"][e], T["Cs"][e])["z"]
                     for e in range(E)], axis=1)


def features(x, T):
    """phi(x) = concat_e [cos z_e, sin z_e], shape (N, 2 E d)."""
    z = phases(x, T)
    N, E, d = z.shape
    return np.concatenate([np.cos(z), np.sin(z)], axis=2).reshape(N, 2 * E * d)


def zhat_matrix(T, e):
    """The explicit d x d matrix Z-hat_e (columns = map applied to basis vectors)."""
    d = T["B"].shape[1]
    eye = np.eye(d)
    return stages(eye, T["B"][e], T["perm"][e], T["G"][e], T["Cs"][e])["z"].T
