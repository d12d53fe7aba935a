"""Mini-batch SGD through the fused forward and the adjoint kernels: the
paper's protocol shape (plain SGD, learning rate 1e-3, batches of 10) on
MNIST-shaped inputs with labels from a fixed linear teacher."""

import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu


def test_sgd_learns_teacher_labels(mck, dev):
    from paper_1702_08159_gb300.autograd import McKernelClassifier
    from paper_1702_08159_gb300.sgd import accuracy, fit

    n, C = 2000, 10
    xh = wl.mnist_like(n, 784, seed=3)
    yh = wl.teacher_labels(xh, C, seed=4)
    x, y = torch.from_numpy(xh).to(dev), torch.from_numpy(yh).to(dev)
    plan = mck.Plan(1024, 4, "rbf", 3.0, 42)
    model = McKernelClassifier(plan, C)  # W = 0, b = 0: loss log(10) at the start
    Cs0, G0 = model.Cs.detach().clone(), model.G.detach().clone()
    acc0 = accuracy(model, x, y)
    hist = fit(model, x, y, lr=1e-3, batch=10, epochs=2, seed=0)
    acc1 = accuracy(model, x, y)
    assert abs(hist[0] - np.log(C)) < 0.5 and hist[1] < hist[0] - 0.2, hist
    assert acc1 > max(0.5, acc0 + 0.3), (acc0, acc1)
    # the calibration and G moved too (they are learnable parameters)
    assert (model.Cs.detach() - Cs0).abs().max().item() > 0
    assert (model.G.detach() - G0).abs().max().item() > 0
    assert all(np.isfinite(hist))


def test_sgd_rejects_bad_labels(mck, dev):
    from paper_1702_08159_gb300.autograd import McKernelClassifier
    from paper_1702_08159_gb300.sgd import fit

    plan = mck.Plan(64, 1, "rbf", 1.0, 1)
    model = McKernelClassifier(plan, 3)
    x = torch.zeros((4, 64), device=dev)
    with pytest.raises(TypeError):
        fit(model, x, torch.zeros(4, dtype=torch.int64, device=dev), epochs=1)
    with pytest.raises(ValueError):
        fit(model, x, torch.zeros(3, dtype=torch.int32, device=dev), epochs=1)
