"""Mini-batch SGD for a McKernel classifier (Sec. "Empirical Analysis": the
feature map feeds softmax(W phi + b), trained with stochastic gradient
descent on the logistic/cross-entropy loss, with the calibration C and the
Gaussian diagonal G learnable as well).

The protocol's shape follows the paper's experiments: plain SGD, learning
rate 1e-3, mini-batches of 10, a fixed number of epochs over a shuffled
training set. Every step runs the fused forward (logits without writing the
features) and the adjoint kernels through ``McKernelClassifier``; the
optimiser update is torch's SGD on the four parameter tensors.
"""

import numpy as np
import torch

from .autograd import McKernelClassifier


def fit(model: McKernelClassifier, x, y, lr=1e-3, batch=10, epochs=20, seed=0, momentum=0.0):
    """Train ``model`` on device tensors x (n, in_dim) float32 and y (n,)
    int32 labels. Returns the mean loss of each epoch (a list of floats; the
    losses are averaged on the device and read once per epoch)."""
    if x.dim() != 2 or y.dim() != 1 or x.shape[0] != y.shape[0]:
        raise ValueError("x must be (n, in_dim) and y (n,)")
    if y.dtype != torch.int32:
        raise TypeError("labels must be int32")
    n = x.shape[0]
    params = [p for p in model.parameters() if p.requires_grad]
    opt = torch.optim.SGD(params, lr=lr, momentum=momentum)
    rng = np.random.default_rng(seed)
    history = []
    for _ in range(epochs):
        order = torch.from_numpy(rng.permutation(n)).to(x.device)
        total = torch.zeros((), device=x.device)
        steps = 0
        for s in range(0, n, batch):
            idx = order[s: s + batch]
            opt.zero_grad(set_to_none=False)
            loss = model.loss(x[idx].contiguous(), y[idx].contiguous())
            loss.backward()
            opt.step()
            total += loss.detach()
            steps += 1
        history.append(float(total.item()) / max(steps, 1))
    return history


@torch.no_grad()
def accuracy(model: McKernelClassifier, x, y, chunk=4096):
    """Fraction of rows whose largest logit is the label."""
    hits = 0
    for s in range(0, x.shape[0], chunk):
        pred = model(x[s: s + chunk].contiguous()).argmax(dim=1)
        hits += int((pred == y[s: s + chunk].long()).sum().item())
    return hits / max(x.shape[0], 1)
