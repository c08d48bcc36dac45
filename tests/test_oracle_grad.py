"""Pins of the oracle's analytic gradient (chain rule through Eqs. 2, 3, 8-10)
against central finite differences of the oracle's own objective, which is
evaluated directly from the definitions (no derivative code involved).

The objective L(alpha) = sum_p c_agg(p, d*(p)) is smooth in alpha except
where a row shift s(v) = alpha0 + alpha1 v - delta crosses an integer (the
linear warp has a kink there), so alpha is chosen with every s(v) at least
ten steps away from an integer, and the alpha1 step is scaled by the lowest
row (a step h1 moves row v by h1 * v pixels).
"""
import numpy as np
import pytest

import oracle
from helpers import kink_free_alpha
from paper_1807_07433_gb300 import synth

H_A0 = 1e-3


def _scene(W=56, H=40, seed=5, D=10):
    w = synth.small(W, H, D=D, ncc_r=2, agg_r=2, seed=seed, alpha0=9.0, alpha1=0.06)
    left, right, _ = synth.make_pair(w.scene)
    return w, left.astype(np.float64), right.astype(np.float64)


def _params(w, a0, a1):
    return oracle.Params(W=w.scene.W, H=w.scene.H, D=w.D, ncc_r=w.ncc_r, agg_r=w.agg_r,
                         gamma_d=w.gamma_d, gamma_r=w.gamma_r, alpha0=a0, alpha1=a1,
                         delta=w.delta)


def _kink_free_alpha(w, h0, h1):
    """alpha near the true plane with every row shift >= 10 steps from an integer."""
    a1 = w.scene.alpha1 + 0.0013
    return kink_free_alpha(w.scene.alpha0 + 0.137, a1, w.delta, w.scene.H, h0, h1), a1


@pytest.mark.parametrize("objective", ["plane", "winning"])
def test_alpha_gradient_matches_central_differences(objective):
    w, left, right = _scene()
    h1 = H_A0 / (w.scene.H - 1)
    a0, a1 = _kink_free_alpha(w, H_A0, h1)
    p = _params(w, a0, a1)
    if objective == "plane":
        dstar = np.full((w.scene.H, w.scene.W), int(w.delta), np.int32)
    else:   # winning labels of the forward pass where the L-R check passed
        res = oracle.match(p, left.astype(np.uint8), right.astype(np.uint8),
                           want=("lbl_l", "valid"))
        dstar = np.where(res.valid.astype(bool), res.lbl_l, -1).astype(np.int32)
    L, da, _, _ = oracle.grad(p, left, right, dstar)
    assert L == pytest.approx(oracle.objective(p, left, right, dstar), rel=1e-12)
    fd0 = (oracle.objective(_params(w, a0 + H_A0, a1), left, right, dstar) -
           oracle.objective(_params(w, a0 - H_A0, a1), left, right, dstar)) / (2 * H_A0)
    fd1 = (oracle.objective(_params(w, a0, a1 + h1), left, right, dstar) -
           oracle.objective(_params(w, a0, a1 - h1), left, right, dstar)) / (2 * h1)
    assert da[0] == pytest.approx(fd0, rel=1e-3)
    assert da[1] == pytest.approx(fd1, rel=1e-3)


def test_image_gradients_match_central_differences():
    w, left, right = _scene(W=40, H=30, seed=9, D=8)
    p = _params(w, w.scene.alpha0 + 0.31, w.scene.alpha1)
    dstar = np.full((w.scene.H, w.scene.W), int(w.delta), np.int32)
    dstar[::3, ::4] = -1                        # a pixel set with holes
    _, _, gl, gr = oracle.grad(p, left, right, dstar)
    rng = np.random.default_rng(0)
    h = 1e-3
    pts = [(0, 0), (w.scene.H - 1, w.scene.W - 1), (5, 0), (0, 7)] + \
        [tuple(x) for x in rng.integers(0, [w.scene.H, w.scene.W], size=(10, 2))]
    for (y, x) in pts:
        for img, g, which in ((left, gl, 0), (right, gr, 1)):
            up, dn = img.copy(), img.copy()
            up[y, x] += h
            dn[y, x] -= h
            args_up = (up, right) if which == 0 else (left, up)
            args_dn = (dn, right) if which == 0 else (left, dn)
            fd = (oracle.objective(p, *args_up, dstar) - oracle.objective(p, *args_dn, dstar)) / (2 * h)
            assert g[y, x] == pytest.approx(fd, rel=1e-3, abs=1e-7), (which, y, x)


def test_plane_objective_peaks_at_true_plane():
    """With the plane hypothesis (every pixel at residual delta), L is largest
    when the warp uses the scene's own alpha (no potholes in this scene)."""
    sc = synth.Scene(64, 48, 10.0, 0.05, 0, False, 21)
    left, right, _ = synth.make_pair(sc)
    w = synth.Workload("plane", sc, D=12, ncc_r=2, agg_r=2, gamma_d=3.0, gamma_r=10.0, delta=5.0)
    dstar = np.full((48, 64), 5, np.int32)
    Ls = {a0: oracle.objective(_params(w, a0, 0.05), left, right, dstar)
          for a0 in (9.0, 9.5, 10.0, 10.5, 11.0)}
    assert max(Ls, key=Ls.get) == 10.0
