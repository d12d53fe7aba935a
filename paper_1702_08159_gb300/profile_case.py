"""A few launches of one workload on seeded synthetic inputs, for profilers.

    python -m paper_1702_08159_gb300.profile_case features --d 1024 --E 16 --rows 15000
    python -m paper_1702_08159_gb300.profile_case logits --d 1024 --E 16 --rows 8192 --classes 10
    python -m paper_1702_08159_gb300.profile_case features --d 16384 --E 4 --rows 2048 --gaussian
    python -m paper_1702_08159_gb300.profile_case logits --d 1024 --E 16 --rows 8192 --prec fp16_split
    python -m paper_1702_08159_gb300.profile_case train --d 1024 --E 16 --rows 512 --classes 10

Inputs: MNIST-shaped rows (784 values, ~80% zeros, others U[0,1), padded to
d) by default, or N(0,1) rows of length d (--gaussian); RBF plan with the
given sigma and seed; --prec selects mck_features_ex / mck_fused_logits_ex
precisions (default fp32); `train` runs the fused training step of the
classifier (forward logits, cross-entropy, the adjoint) on uniform random
labels. The workload runs `--launches` times (default 3, the
first a warm-up) with the plan's automatic launch shape, then the process
synchronises and prints one line. Under ncu, `-k regex:<kernel> -s 1 -c 1`
captures the second launch.
"""

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("what", choices=["features", "logits", "train"])
    p.add_argument("--d", type=int, default=1024)
    p.add_argument("--E", type=int, default=16)
    p.add_argument("--rows", type=int, default=8192)
    p.add_argument("--classes", type=int, default=10)
    p.add_argument("--sigma", type=float, default=3.0)
    p.add_argument("--seed", type=int, default=42)
    p.add_argument("--gaussian", action="store_true")
    p.add_argument("--launches", type=int, default=3)
    p.add_argument("--prec", default="fp32")
    a = p.parse_args(argv)

    import torch

    import paper_1702_08159_gb300 as mck
    import workloads as wl

    plan = mck.Plan(a.d, a.E, "rbf", a.sigma, a.seed)
    xh = wl.gaussian(a.rows, a.d, seed=a.seed) if a.gaussian else wl.mnist_like(a.rows, min(784, a.d), seed=a.seed)
    x = torch.from_numpy(xh).cuda()
    if a.what == "features":
        out = torch.empty((a.rows, plan.num_features), device="cuda")
        for _ in range(a.launches):
            mck.features(plan, x, out=out, prec=a.prec)
    elif a.what == "logits":
        W, b = wl.logit_weights(a.classes, plan.num_features, seed=a.seed)
        Wd, bd = torch.from_numpy(W).cuda(), torch.from_numpy(b).cuda()
        out = torch.empty((a.rows, a.classes), device="cuda")
        for _ in range(a.launches):
            mck.fused_logits(plan, x, Wd, bd, out=out, prec=a.prec)
    else:
        from paper_1702_08159_gb300.autograd import McKernelClassifier

        W, b = wl.logit_weights(a.classes, plan.num_features, seed=a.seed)
        model = McKernelClassifier(plan, a.classes, torch.from_numpy(W), torch.from_numpy(b))
        y = torch.from_numpy(wl.labels(a.rows, a.classes, seed=a.seed)).cuda()
        for _ in range(a.launches):
            for q in model.parameters():
                q.grad = None
            model.loss(x, y).backward()
        out = model.W.grad
    torch.cuda.synchronize()
    print(f"profile_case {a.what} d={a.d} E={a.E} rows={a.rows} prec={a.prec}: ok ({float(out[0, :4].sum()):.6f})")
    plan.close()


if __name__ == "__main__":
    main()
