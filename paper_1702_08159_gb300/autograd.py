"""torch.autograd wrappers around the library's forward and adjoint kernels.

Sec. "Empirical Analysis and Experiments" trains softmax(W phi + b) by SGD
and proposes learning the calibration C and G by backpropagation, and
learning B (likened there to attention). These Functions expose the
hand-written adjoint (H^T = H, Pi^T = Pi^{-1}, forward recomputed instead of
stored) to autograd.

Learned signs: B stays a +-1 diagonal in every kernel. A trainer keeps a
real-valued latent B_r (E x d); each forward first sets the plan's signs to
sign(B_r) (``Plan.set_signs``, negative -> -1), and the backward returns the
straight-through gradient of Bengio, Leonard and Courville (2013) with the
hard-tanh gate of BinaryConnect (Courbariaux et al., 2015): the exact
gradient with respect to B read as a real diagonal (the map is linear in B,
u0 = B x-hat), kept where |B_r| <= 1 and zeroed elsewhere. Pi stays fixed.
"""

import torch

from . import features, features_backward, fused_logits, fused_logits_backward, softmax_xent


def _straight_through(dB, Br):
    """dB where |B_r| <= 1, zero elsewhere (the hard-tanh gate)."""
    return dB * (Br.abs() <= 1).to(dB.dtype)


class FastfoodFeatures(torch.autograd.Function):
    """phi = features(plan, x, Cs, G), with the plan's signs set to sign(Br)
    first when a latent Br is given; gradients for x, Cs, G (and Br)."""

    @staticmethod
    def forward(ctx, plan, x, Cs, G, Br=None):
        ctx.plan = plan
        if Br is not None:
            plan.set_signs(Br)
        ctx.save_for_backward(x, Cs, G, Br)
        return features(plan, x, Cs, G)

    @staticmethod
    def backward(ctx, dphi):
        x, Cs, G, Br = ctx.saved_tensors
        nx, nc, ng = ctx.needs_input_grad[1:4]
        nB = Br is not None and ctx.needs_input_grad[4]
        if Br is not None:
            ctx.plan.set_signs(Br)  # the signs this forward used
        r = features_backward(ctx.plan, x, dphi, Cs, G, need_dx=nx, need_dCs=nc, need_dG=ng,
                              need_dB=nB)
        dBr = _straight_through(r[3], Br) if nB else None
        return (None, r[0], r[1], r[2]) + ((dBr,) if len(ctx.needs_input_grad) > 4 else ())


class FastfoodLogits(torch.autograd.Function):
    """logits = W phi(x) + b with phi never materialised, with the plan's signs
    set to sign(Br) first when a latent Br is given; gradients for x, Cs, G,
    W, b (and Br)."""

    @staticmethod
    def forward(ctx, plan, x, Cs, G, W, b, Br=None):
        ctx.plan = plan
        if Br is not None:
            plan.set_signs(Br)
        ctx.save_for_backward(x, Cs, G, W, Br)
        ctx.has_b = b is not None
        return fused_logits(plan, x, W, b, Cs, G)

    @staticmethod
    def backward(ctx, dlogits):
        x, Cs, G, W, Br = ctx.saved_tensors
        nx, nc, ng, nw, nb = ctx.needs_input_grad[1:6]
        nB = Br is not None and ctx.needs_input_grad[6]
        if Br is not None:
            ctx.plan.set_signs(Br)  # the signs this forward used
        g = fused_logits_backward(ctx.plan, x, W, dlogits.contiguous(), Cs, G, need_dx=nx,
                                  need_dCs=nc, need_dG=ng, need_dW=nw, need_db=nb and ctx.has_b,
                                  need_dB=nB)
        dBr = _straight_through(g["dB"], Br) if nB else None
        out = (None, g["dx"], g["dCs"], g["dG"], g["dW"], g["db"])
        return out + ((dBr,) if len(ctx.needs_input_grad) > 6 else ())


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
    """softmax(W phi(x) + b) with learnable Cs and G (initialised from the plan)
    and, with ``learn_signs``, a latent Br (initialised to the plan's signs)
    whose signs become B at every forward.

    ``forward`` returns logits; ``loss`` the mean cross-entropy. The feature
    map runs fused with the logits (phi is never written to memory). With
    learned signs the plan's B is overwritten at each forward: a plan is
    then owned by one classifier.
    """

    def __init__(self, plan, num_classes, W=None, b=None, learn_calibration=True,
                 learn_signs=False):
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
        self.Br = (torch.nn.Parameter(torch.from_numpy(plan.signs()).to(dev))
                   if learn_signs else None)

    def forward(self, x):
        return FastfoodLogits.apply(self.plan, x, self.Cs, self.G, self.W, self.b, self.Br)

    def loss(self, x, labels):
        return SoftmaxCrossEntropy.apply(self(x), labels)
