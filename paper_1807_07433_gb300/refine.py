"""Road-plane refinement by gradient ascent on the aggregated matching cost.

The paper estimates the Eq. 2 plane once, by least squares on a disparity
map (Sec. II-A).  Here the plane is refined against the images themselves:
with the disparities of a pixel set held fixed (the plane hypothesis puts
every pixel at residual delta, i.e. full disparity alpha0 + alpha1 v), the
objective is

    L(alpha) = sum_p c_agg(p, dstar[p])          (Eq. 8 over Eq. 3, Sec. II-A warp)

and its gradient comes from the hand-written adjoint behind sr_grad_plane
(include/sr.h).  `PlaneCost` wraps that adjoint as a torch.autograd.Function;
`refine_plane` runs L-BFGS (or Adam) on it.

The loop is generic over the evaluator (any object with
value_and_grad(alpha0, alpha1) -> (L, dL/dalpha), optionally n_pixels);
`MatcherEvaluator` is the CUDA one.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch


class PlaneCost(torch.autograd.Function):
    """L(alpha) as a differentiable function of alpha = (alpha0, alpha1).

    Forward makes one call that returns both L and dL/dalpha (the adjoint
    reuses everything the objective computes); backward scales the stored
    gradient.  alpha is a float64 CPU tensor of shape (2,)."""

    @staticmethod
    def forward(ctx, alpha, evaluator):
        a = alpha.detach().to("cpu", torch.float64)
        L, g = evaluator.value_and_grad(float(a[0]), float(a[1]))
        ctx.save_for_backward(torch.as_tensor(np.asarray(g, np.float64), dtype=alpha.dtype))
        return alpha.new_tensor(float(L))

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g.to(grad_out.device), None


class MatcherEvaluator:
    """value_and_grad on the CUDA path: sr_set_plane + sr_grad_plane."""

    def __init__(self, matcher, left, right, dstar, delta):
        self.m, self.left, self.right, self.dstar = matcher, left, right, dstar
        self.delta = float(delta)
        self.n_pixels = int(dstar.numel())

    def value_and_grad(self, alpha0, alpha1):
        self.m.set_plane(alpha0, alpha1, self.delta)
        return self.m.grad_plane(self.left, self.right, self.dstar)


@dataclass
class RefineResult:
    alpha: tuple
    history: list = field(default_factory=list)   # (alpha0, alpha1, L) per evaluation


class _Recorder:
    """Counts evaluations and records (alpha0, alpha1, L) for each."""

    def __init__(self, evaluator, res):
        self.ev, self.res = evaluator, res

    def value_and_grad(self, a0, a1):
        L, g = self.ev.value_and_grad(a0, a1)
        self.res.history.append((a0, a1, float(L)))
        return L, g


def refine_plane(evaluator, alpha_init, H, max_evals=50, method="lbfgs", lr=1.0,
                 lr_final=0.02) -> RefineResult:
    """Maximise L from alpha_init within max_evals evaluations of L and its
    gradient.  The parameters are theta = (shift at the middle row, shift
    change from the first to the last row), both in pixels: centring the row
    index decouples the two directions of the Eq. 2 plane.

    method "lbfgs": L-BFGS with a strong-Wolfe line search on -L / (pixel
    count); "adam": Adam with a cosine-decayed learning rate lr -> lr_final
    (pixels of theta), one evaluation per step.  Returns the best alpha seen
    and the history of every evaluation."""
    c = (H - 1) / 2.0
    theta = torch.tensor([alpha_init[0] + alpha_init[1] * c, alpha_init[1] * (H - 1)],
                         dtype=torch.float64, requires_grad=True)
    res = RefineResult(alpha=tuple(alpha_init))
    ev = _Recorder(evaluator, res)

    def alpha_of(t):
        a1 = t[1] / (H - 1)
        return torch.stack([t[0] - a1 * c, a1])

    if method == "lbfgs":
        opt = torch.optim.LBFGS([theta], lr=1.0, max_iter=max_evals, max_eval=max_evals,
                                history_size=10, tolerance_grad=1e-12, tolerance_change=1e-14,
                                line_search_fn="strong_wolfe")
        scale = 1.0 / float(getattr(evaluator, "n_pixels", H))

        def closure():
            opt.zero_grad()
            loss = -PlaneCost.apply(alpha_of(theta), ev) * scale
            loss.backward()
            return loss
        opt.step(closure)
    elif method == "adam":
        opt = torch.optim.Adam([theta], lr=lr, maximize=True)
        for k in range(max_evals):
            for grp in opt.param_groups:
                grp["lr"] = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * k / max_evals))
            opt.zero_grad()
            PlaneCost.apply(alpha_of(theta), ev).backward()
            opt.step()
    else:
        raise ValueError(f"unknown method {method!r}")
    best = max(res.history, key=lambda h: h[2])
    res.alpha = (best[0], best[1])
    return res
