"""Host logic of the plane refinement (PlaneCost autograd.Function and the
Adam loop), driven on the CPU by the FP64 oracle as the evaluator."""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_07433_gb300 import refine, synth


class OracleEvaluator:
    def __init__(self, w, left, right, dstar):
        self.w = w
        self.l, self.r = left.astype(np.float64), right.astype(np.float64)
        self.d = dstar.astype(np.int32)
        self.n_pixels = self.d.size
        self.calls = 0

    def value_and_grad(self, a0, a1):
        w = self.w
        self.calls += 1
        p = oracle.Params(W=w.scene.W, H=w.scene.H, D=w.D, ncc_r=w.ncc_r, agg_r=w.agg_r,
                          gamma_d=w.gamma_d, gamma_r=w.gamma_r, alpha0=a0, alpha1=a1,
                          delta=w.delta)
        L, da, _, _ = oracle.grad(p, self.l, self.r, self.d)
        return L, da


def _scene(W=96, H=64):
    sc = synth.Scene(W, H, 20.0, 0.03, 0, False, 11)
    w = synth.Workload("refine", sc, D=16, ncc_r=3, agg_r=3, gamma_d=3.0, gamma_r=10.0,
                       delta=8.0)
    left, right, _ = synth.make_pair(sc)
    return w, left, right, np.full((H, W), 8, np.int32)


def test_plane_cost_backward_returns_scaled_gradient():
    w, left, right, dstar = _scene(48, 32)
    ev = OracleEvaluator(w, left, right, dstar)
    alpha = torch.tensor([20.3, 0.031], dtype=torch.float64, requires_grad=True)
    L = refine.PlaneCost.apply(alpha, ev)
    (3.0 * L).backward()
    L_ref, g_ref = ev.value_and_grad(20.3, 0.031)
    assert float(L.detach()) == pytest.approx(L_ref, rel=1e-15)
    np.testing.assert_allclose(alpha.grad.numpy(), 3.0 * np.asarray(g_ref), rtol=1e-15)


@pytest.mark.parametrize("method,evals", [("lbfgs", 30), ("adam", 40)])
def test_refinement_reaches_the_maximum_of_L(method, evals):
    """From a perturbed plane, refinement ends at least as high as the scene's
    own plane (the maximum of L sits within noise of it) and within 0.3 px."""
    w, left, right, dstar = _scene()
    ev = OracleEvaluator(w, left, right, dstar)
    sc = w.scene
    rng = np.random.default_rng(5)
    a_init = (sc.alpha0 + rng.uniform(-1.5, 1.5), sc.alpha1 + rng.uniform(-0.01, 0.01))
    res = refine.refine_plane(ev, a_init, sc.H, max_evals=evals, method=method)
    assert ev.calls == len(res.history) <= evals + 1
    L_true = ev.value_and_grad(sc.alpha0, sc.alpha1)[0]
    L_final = max(h[2] for h in res.history)
    assert (res.alpha[0], res.alpha[1], L_final) in res.history
    assert L_final >= L_true - 1e-6 * abs(L_true)
    assert abs(res.alpha[0] - sc.alpha0) < 0.3
    assert abs(res.alpha[1] - sc.alpha1) * (sc.H - 1) < 0.3


def test_unknown_method_is_rejected():
    with pytest.raises(ValueError):
        refine.refine_plane(None, (1.0, 0.0), 10, method="sgd")
