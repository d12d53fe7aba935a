"""Mini-batch SGD for a McKernel classifier (Sec. "Empirical Analysis": the
feature map feeds softmax(W phi + b), trained with stochastic gradient
descent on the logistic/cross-entropy loss, with the calibration C and the
Gaussian diagonal G learnable as well).

The protocol's shape follows the paper's experiments: plain SGD, learning
rate 1e-3, mini-batches of 10, a fixed number of epochs over a shuffled
training set. Every step runs the fused forward (logits without writing the
features) and the adjoint kernels through ``McKernelClassifier``; the
optimiser update is torch's SGD on the four parameter tensors.

Data parallel (Sec. "Large-scale Machine Learning": the hashed parameters
are the same on every machine): with torch.distributed initialised and more
than one rank, every rank draws the same shuffled order, takes its
contiguous share of each global mini-batch, weights its mean loss by its
share, and the gradients are summed over ranks before the update, so every
rank applies the update of the global mini-batch and the replicas stay equal.
"""

import numpy as np
import torch
import torch.distributed as dist

from .autograd import McKernelClassifier
from .dist import allreduce_grads, shard_range


def _world():
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def fit(model: McKernelClassifier, x, y, lr=1e-3, batch=10, epochs=20, seed=0, momentum=0.0):
    """Train ``model`` on device tensors x (n, in_dim) float32 and y (n,)
    int32 labels (every rank holds the same x and y when data parallel).
    Returns the mean loss of each epoch over the global mini-batches (a list
    of floats; the losses are averaged on the device and read once per
    epoch)."""
    if x.dim() != 2 or y.dim() != 1 or x.shape[0] != y.shape[0]:
        raise ValueError("x must be (n, in_dim) and y (n,)")
    if y.dtype != torch.int32:
        raise TypeError("labels must be int32")
    n = x.shape[0]
    rank, world = _world()
    params = [p for p in model.parameters() if p.requires_grad]
    for p in params:  # every rank then all-reduces the same tensors, even for an empty share
        if p.grad is None:
            p.grad = torch.zeros_like(p)
    opt = torch.optim.SGD(params, lr=lr, momentum=momentum)
    rng = np.random.default_rng(seed)
    history = []
    for _ in range(epochs):
        order = torch.from_numpy(rng.permutation(n)).to(x.device)
        total = torch.zeros((), dtype=torch.float64, device=x.device)
        steps = 0
        for s in range(0, n, batch):
            idx = order[s: s + batch]
            if world > 1:
                lo, hi = shard_range(len(idx), rank, world)
                share = (hi - lo) / len(idx)
                idx = idx[lo:hi]
            else:
                share = 1.0
            opt.zero_grad(set_to_none=False)
            if len(idx):
                loss = model.loss(x[idx].contiguous(), y[idx].contiguous()) * share
                loss.backward()
                total += loss.detach()
            if world > 1:
                allreduce_grads(params)
            opt.step()
            steps += 1
        if world > 1:
            dist.all_reduce(total, op=dist.ReduceOp.SUM)
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
