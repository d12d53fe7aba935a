"""torch.autograd wrappers around the library's forward and adjoint kernels.

Sec. "Empirical Analysis and Experiments" trains softmax(W phi + b) by SGD
and proposes learning the calibration C and G by backpropagation. These
Functions expose the hand-written adjoint (H^T = H, Pi^T = Pi^{-1}, forward
recomputed instead of stored) to autograd. B and Pi stay fixed (they come
from the plan's hash).
"""

import torch

from . import features, features_backward, fused_logits, fused_logits_backward, softmax_xent


class FastfoodFeatures(torch.autograd.Function):
    """phi = features(plan, x, Cs, G); gradients for x, Cs and G."""

    @staticmethod
    def forward(ctx, plan, x, Cs, G):
        ctx.plan = plan
        ctx.save_for_backward(x, Cs, G)
        return features(plan, x, Cs, G)

    @staticmethod
    def backward(ctx, dphi):
        x, Cs, G = ctx.saved_tensors
        nx, nc, ng = ctx.needs_input_grad[1:4]
        dx, dCs, dG = features_backward(ctx.plan, x, dphi, Cs, G, need_dx=nx, need_dCs=nc,
                                        need_dG=ng)
        return None, dx, dCs, dG


class FastfoodLogits(torch.autograd.Function):
    """logits = W phi(x) + b with phi never materialised; gradients for x, Cs, G, W, b."""

    @staticmethod
    def forward(ctx, plan, x, Cs, G, W, b):
        ctx.plan = plan
        ctx.save_for_backward(x, Cs, G, W)
        ctx.has_b = b is not None
        return fused_logits(plan, x, W, b, Cs, G)

    @staticmethod
    def backward(ctx, dlogits):
        x, Cs, G, W = ctx.saved_tensors
        nx, nc, ng, nw, nb = ctx.needs_input_grad[1:6]
        g = fused_logits_backward(ctx.plan, x, W, dlogits.contiguous(), Cs, G, need_dx=nx,
                                  need_dCs=nc, need_dG=ng, need_dW=nw, need_db=nb and ctx.has_b)
        return None, g["dx"], g["dCs"], g["dG"], g["dW"], g["db"]


class SoftmaxCrossEntropy(torch.autograd.Function):
    """Mean softmax cross-entropy (multi-class form of Eq. etn:loss)."""

    @staticmethod
    def forward(ctx, logits, labels):
        loss, dl = softmax_xent(logits, labels, need_grad=True)
        ctx.save_for_backward(dl)
        return loss

    @staticmethod
    def backward(ctx, dloss):
        (dl,) = ctx.saved_tensors
        return dl * dloss, None


class McKernelClassifier(torch.nn.Module):
    """softmax(W phi(x) + b) with learnable Cs and G (initialised from the plan).

    ``forward`` returns logits; ``loss`` the mean cross-entropy. The feature
    map runs fused with the logits (phi is never written to memory).
    """

    def __init__(self, plan, num_classes, W=None, b=None, learn_calibration=True):
        super().__init__()
        self.plan = plan
        t = plan.tables()
        dev = torch.device("cuda", plan.device)
        self.Cs = torch.nn.Parameter(torch.from_numpy(t["Cs"]).to(dev),
                                     requires_grad=learn_calibration)
        self.G = torch.nn.Parameter(torch.from_numpy(t["G"]).to(dev),
                                    requires_grad=learn_calibration)
        F = plan.num_features
        W = torch.zeros(num_classes, F) if W is None else torch.as_tensor(W)
        b = torch.zeros(num_classes) if b is None else torch.as_tensor(b)
        self.W = torch.nn.Parameter(W.to(dev, torch.float32).contiguous())
        self.b = torch.nn.Parameter(b.to(dev, torch.float32).contiguous())

    def forward(self, x):
        return FastfoodLogits.apply(self.plan, x, self.Cs, self.G, self.W, self.b)

    def loss(self, x, labels):
        return SoftmaxCrossEntropy.apply(self(x), labels)
