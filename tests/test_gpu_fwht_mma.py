"""Tensor-core Kronecker-H16 transform (mck_fwht with 16-bit precisions) against the oracle.

Error model, relative to sqrt(d) rms(x) (the size of an output): each 16-bit
rounding of an operand has relative error <= 2^-p (p = 8 for bf16, 11 for fp16
with round-to-nearest: half an ulp of a p+1-bit significand); an unsplit
transform rounds twice (the input and the intermediate after the first digit),
so errors stay near 2^-p; the hi + lo split leaves 2^-2p per rounding. The
BOUND values allow a factor of 4 to 8 over those sizes, far below the O(1)
error of any wrong index or sign: they are regression bounds of the error
model, one per form, not the accuracy target.

The accuracy target for the 16-bit forms is a max abs error of 2e-3 on the
orthonormal output (error relative to sqrt(d) rms(x), as measured here).
FP16 unsplit and both hi + lo forms meet it (test_accuracy_target).
BF16 unsplit does NOT meet it: rounding the input to 8 significant bits alone
leaves 2^-9 relative error per element, about 1.1e-3 rms after the transform
and ~5e-3 at the maximum over millions of outputs (1.2e-2 measured at
d = 1024). No test claims that bar for BF16 unsplit.
"""

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import fastfood as ff

pytestmark = pytest.mark.gpu

# Error-model regression bounds (see the module docstring), not the target.
BOUND = {"bf16": 2.0 ** -6, "fp16": 2.0 ** -8, "bf16_split": 2.0 ** -14, "fp16_split": 2.0 ** -18}
# The target's max abs error for the 16-bit forms; BF16 unsplit is excluded
# because it cannot meet it (module docstring).
TARGET_BAR = 2e-3
MEETS_BAR = ("fp16", "bf16_split", "fp16_split")


def _rel_err(got, x):
    d = x.shape[1]
    return float(np.abs(got.astype(np.float64) - ff.fwht(x.astype(np.float64))).max()
                 / (np.sqrt(d) * np.sqrt((x.astype(np.float64) ** 2).mean())))


@pytest.mark.parametrize("prec", list(BOUND))
@pytest.mark.parametrize("d", [256, 512, 1024])
def test_tensor_core_transform_accuracy(mck, dev, d, prec):
    n = (4096 // d) * 3
    x = wl.gaussian(n, d, seed=d)
    t = torch.from_numpy(x).to(dev)
    mck.fwht_(t, prec)
    err = _rel_err(t.cpu().numpy(), x)
    assert err <= BOUND[prec], (d, prec, err)


@pytest.mark.parametrize("prec", list(BOUND))
@pytest.mark.parametrize("L,n", [(11, 3), (13, 2), (15, 1), (16, 1), (18, 1), (20, 1)])
def test_tensor_core_large_d(mck, dev, L, n, prec):
    # d > 1024: tensor cores on every 1024-float block, FP32 column passes above
    d = 1 << L
    x = wl.gaussian(n, d, seed=L)
    t = torch.from_numpy(x).to(dev)
    mck.fwht_(t, prec)
    err = _rel_err(t.cpu().numpy(), x)
    assert err <= BOUND[prec], (d, prec, err)


@pytest.mark.parametrize("prec", ["bf16", "fp16_split"])
def test_tensor_core_basis_vectors_exact_d4096(mck, dev, prec):
    d = 4096
    t = torch.eye(d, device=dev)
    mck.fwht_(t, prec)
    np.testing.assert_array_equal(t.cpu().numpy(), ff.sylvester(d))


@pytest.mark.parametrize("prec", list(BOUND))
def test_tensor_core_basis_vectors_exact(mck, dev, prec):
    # H e_i is a row of the Sylvester matrix: +-1 values, exact in every precision.
    d = 1024
    t = torch.eye(d, device=dev)
    mck.fwht_(t, prec)
    np.testing.assert_array_equal(t.cpu().numpy(), ff.sylvester(d))


def test_split_is_more_accurate(mck, dev):
    x = wl.gaussian(64, 1024, seed=3)
    errs = {}
    for prec in ("bf16", "bf16_split", "fp16", "fp16_split"):
        t = torch.from_numpy(x).to(dev)
        mck.fwht_(t, prec)
        errs[prec] = _rel_err(t.cpu().numpy(), x)
    assert errs["bf16_split"] < errs["bf16"] / 64
    assert errs["fp16_split"] < errs["fp16"] / 64
    assert errs["fp16"] < errs["bf16"]


def test_tensor_core_rejects_unsupported_shapes(mck, dev):
    with pytest.raises(mck.MckError, match="UNSUPPORTED"):
        mck.fwht_(torch.zeros((8, 128), device=dev), "bf16")
    with pytest.raises(mck.MckError, match="multiple of 1024"):
        mck.fwht_(torch.zeros((3, 256), device=dev), "bf16")


@pytest.mark.parametrize("prec", MEETS_BAR)
@pytest.mark.parametrize("L,n", [(10, 4096), (14, 256), (20, 4)])
def test_accuracy_target(mck, dev, L, n, prec):
    """The 2e-3 max abs error target on many outputs (2^22 at d = 1024 and
    2^14, 2^22 at 2^20) for the forms that meet it."""
    d = 1 << L
    x = wl.gaussian(n, d, seed=100 + L)
    t = torch.from_numpy(x).to(dev)
    mck.fwht_(t, prec)
    err = _rel_err(t.cpu().numpy(), x)
    assert err <= TARGET_BAR, (d, prec, err)
