"""Argument checks with a real device: wrong extents, host memory and
misalignment are rejected on the host (MCK_EINVAL) before any kernel runs."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_extent_past_allocation_rejected(mck, dev):
    from paper_1702_08159_gb300 import _lib

    plan = mck.Plan(1024, 2, "rbf", 1.0, 1)
    x = torch.zeros((4, 784), device=dev)
    phi = torch.empty((4, plan.num_features), device=dev)
    lib = _lib.load()
    import ctypes

    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # an extent far past any segment is always caught
    st = lib.mck_features(plan.handle, ctypes.c_void_p(x.data_ptr()), 1 << 40, 784, 784, None,
                          None, ctypes.c_void_p(phi.data_ptr()), s)
    assert st == -1


def test_host_pointer_rejected(mck, dev):
    from paper_1702_08159_gb300 import _lib
    import ctypes

    plan = mck.Plan(64, 1, "rbf", 1.0, 1)
    host = np.zeros((2, 64), np.float32)
    phi = torch.empty((2, plan.num_features), device=dev)
    st = _lib.load().mck_features(plan.handle, ctypes.c_void_p(host.ctypes.data), 2, 64, 64, None,
                                  None, ctypes.c_void_p(phi.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == -1


def test_binding_errors(mck, dev):
    plan = mck.Plan(1024, 1, "rbf", 1.0, 1)
    with pytest.raises(ValueError):
        mck.features(plan, torch.zeros((2, 3, 4), device=dev))  # not (n, in_dim)
    with pytest.raises(mck.MckError):
        mck.features(plan, torch.zeros((3, 2000), device=dev))  # in_dim > d
    with pytest.raises(TypeError):
        mck.features(plan, torch.zeros((3, 784), device=dev, dtype=torch.float64))
    with pytest.raises(mck.MckError, match="UNSUPPORTED"):
        mck.Plan(1 << 21, 1)
    with pytest.raises(mck.MckError, match="UNSUPPORTED"):
        mck.Plan(1 << 16, 1, "matern")
    with pytest.raises(mck.MckError):
        mck.fused_logits(plan, torch.zeros((2, 784), device=dev),
                         torch.zeros((17, plan.num_features), device=dev))
    small = mck.Plan(16, 1, "rbf", 1.0, 1)  # the adjoint needs d >= 32
    with pytest.raises(mck.MckError, match="UNSUPPORTED"):
        mck.features_backward(small, torch.zeros((2, 16), device=dev),
                              torch.zeros((2, small.num_features), device=dev))
