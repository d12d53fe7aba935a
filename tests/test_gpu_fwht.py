"""Standalone transform (mck_fwht) against the oracle's Hadamard recursion.

Tolerance: each output is a sum of d terms formed by L = log2 d rounded
float32 additions; the forward error is below L * 2^-24 * sum|x_j|, and for
random inputs its typical size is sqrt(L/3) 2^-24 sqrt(d) rms(x). The bound
used here, max|err| <= L 2^-21 sqrt(d) rms(x), sits well above rounding and
far below any wrong index or sign (which moves an output by O(sqrt(d) rms(x))).
"""

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import fastfood as ff

pytestmark = pytest.mark.gpu


def _check(got, x64):
    d = x64.shape[-1]
    L = max(1, d.bit_length() - 1)
    ref = ff.fwht(x64)
    scale = np.sqrt(d) * np.sqrt((x64 ** 2).mean())
    err = np.abs(got.astype(np.float64) - ref).max()
    assert err <= L * 2.0 ** -21 * scale, (d, err, scale)


@pytest.mark.parametrize("L", list(range(0, 16)))
@pytest.mark.parametrize("n", [1, 7, 33])
def test_fwht_one_pass_sizes(mck, dev, L, n):
    d = 1 << L
    x = wl.gaussian(n, d, seed=L * 100 + n)
    t = torch.from_numpy(x).to(dev)
    mck.fwht_(t)
    _check(t.cpu().numpy(), x.astype(np.float64))


@pytest.mark.parametrize("L,n", [(16, 3), (17, 2), (18, 1), (19, 1), (20, 2)])
def test_fwht_large_sizes(mck, dev, L, n):
    d = 1 << L
    x = wl.gaussian(n, d, seed=L)
    t = torch.from_numpy(x).to(dev)
    mck.fwht_(t)
    _check(t.cpu().numpy(), x.astype(np.float64))


@pytest.mark.parametrize("L", [10, 13, 20])
def test_fwht_twice_is_d_identity(mck, dev, L):
    d = 1 << L
    x = wl.gaussian(4 if L < 20 else 1, d, seed=5)
    t = torch.from_numpy(x).to(dev)
    mck.fwht_(mck.fwht_(t))
    got = t.cpu().numpy().astype(np.float64) / d
    assert np.abs(got - x).max() < 2 * L * 2.0 ** -21 * np.abs(x).max()


def test_fwht_basis_vectors_exact(mck, dev):
    # H e_i is row i of the Sylvester matrix: exact in float32.
    d = 64
    t = torch.eye(d, device=dev)
    mck.fwht_(t)
    np.testing.assert_array_equal(t.cpu().numpy(), ff.sylvester(d))


@pytest.mark.parametrize("L", [14, 16, 17, 20])
def test_fwht_config2_batch_sampled(mck, dev, L):
    # The sweep's batch shape (1 GiB of float32), checked on sampled rows: at
    # d = 2^16 and 2^17 the clusters loop over many vectors (one pass through
    # distributed shared memory), at 2^20 two passes over HBM.
    d = 1 << L
    n = (1 << 28) // d
    host = wl.gaussian(n, d, seed=42)
    x = torch.from_numpy(host).to(dev)
    rows = [0, 1, n // 2, n - 1]
    before = host[rows].astype(np.float64)
    del host
    mck.fwht_(x)
    torch.cuda.synchronize()
    _check(x[rows].cpu().numpy(), before)


def test_fwht_empty_and_trivial(mck, dev):
    t = torch.empty((0, 1024), device=dev)
    mck.fwht_(t)
    one = torch.tensor([[3.5]], device=dev)
    mck.fwht_(one)
    assert one.item() == 3.5
