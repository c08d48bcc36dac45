"""GPU adjoint (sr_grad_plane) against the FP64 oracle gradient and against
central differences of the GPU's own objective.

Tolerances (FP32 terms, FP64 sums):
  L        |L_gpu - L_orc| <= TOL_AGG * (pixels in the set): each pixel's
           c_agg carries at most the aggregated-cost error of the forward path
  dL/dalpha  rel 1e-3, against the oracle's analytic gradient and against
           central differences (of the oracle's FP64 objective, and of the
           GPU's own): per-term FP32 error ~1e-6 relative; the sum cancels
           (terms of both signs), so alpha is taken off the optimum where the
           gradient is large (measured: <= 3e-6 against the oracle, 1.3e-5
           against the GPU's FP32 differences)
  images   |g_gpu - g_orc| <= 2e-3 |g_orc| + 1e-3 max|g_orc|
"""
import numpy as np
import pytest

from helpers import TOL_AGG, kink_free_alpha, oracle_params
from paper_1807_07433_gb300 import synth

pytestmark = pytest.mark.gpu


def _gpu_grad(w, left, right, dstar, a0, a1, image_grads=True):
    import torch
    from paper_1807_07433_gb300 import sr
    H, W = left.shape
    with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r,
                    stream=torch.cuda.current_stream()) as m:
        m.set_plane(a0, a1, w.delta)
        ds = torch.from_numpy(dstar.astype(np.int16)).cuda()
        r = m.grad_plane(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(), ds,
                         image_grads=image_grads)
        if image_grads:
            return r[0], r[1], r[2].cpu().numpy(), r[3].cpu().numpy()
        return r


def _orc_grad(w, left, right, dstar, a0, a1):
    import oracle
    p = oracle_params(w)
    p.alpha0, p.alpha1 = a0, a1
    return oracle.grad(p, left.astype(np.float64), right.astype(np.float64),
                       np.where((dstar >= 0) & (dstar < w.D), dstar, -1).astype(np.int32))


def _check(w, left, right, dstar, a0, a1):
    L, da, gl, gr = _gpu_grad(w, left, right, dstar, a0, a1)
    Lo, dao, glo, gro = _orc_grad(w, left, right, dstar, a0, a1)
    n_set = int(((dstar >= 0) & (dstar < w.D)).sum())
    assert abs(L - Lo) <= TOL_AGG * max(n_set, 1), (L, Lo)
    np.testing.assert_allclose(da, dao, rtol=1e-3, atol=1e-9)
    for g, go in ((gl, glo), (gr, gro)):
        tol = 2e-3 * np.abs(go) + 1e-3 * max(np.abs(go).max(), 1e-12)
        bad = np.abs(g - go) > tol
        assert not bad.any(), (np.argwhere(bad)[:5], g[bad][:5], go[bad][:5])


PLANE_CASES = [
    synth.C1,                                                    # 160x120 D16 ncc5 bil9
    synth.small(203, 77, D=32, ncc_r=3, agg_r=5, seed=11),       # ragged
    synth.small(70, 38, D=64, ncc_r=5, agg_r=2, seed=13, alpha1=0.11),
    synth.small(33, 5, D=16, ncc_r=2, agg_r=3, seed=14),         # fewer rows than the window
]


@pytest.mark.parametrize("w", PLANE_CASES, ids=lambda w: w.name)
def test_plane_objective_matches_oracle(w):
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    dstar = np.full((H, W), int(w.delta), np.int16)
    dstar[::5, ::3] = -1                                         # holes in the pixel set
    _check(w, left, right, dstar, w.scene.alpha0 + 0.37, w.scene.alpha1 - 0.002)


def test_winning_objective_matches_oracle():
    import oracle
    w = synth.small(150, 90, D=32, ncc_r=3, agg_r=4, seed=21)
    left, right, _ = synth.make_pair(w.scene)
    res = oracle.match(oracle_params(w), left, right, want=("lbl_l", "valid"))
    dstar = np.where(res.valid.astype(bool), res.lbl_l, -1).astype(np.int16)
    _check(w, left, right, dstar, w.scene.alpha0 - 0.23, w.scene.alpha1 + 0.001)


def test_out_of_range_labels_are_left_out():
    w = synth.small(64, 48, D=16, ncc_r=2, agg_r=3, seed=22)
    left, right, _ = synth.make_pair(w.scene)
    rng = np.random.default_rng(3)
    dstar = rng.integers(-3, w.D + 3, size=left.shape).astype(np.int16)
    dstar[0, :4] = (16, 300, -32768, 32767)
    _check(w, left, right, dstar, w.scene.alpha0 + 0.11, w.scene.alpha1)
    L, _ = _gpu_grad(w, left, right, np.full(left.shape, -1, np.int16), w.scene.alpha0,
                     w.scene.alpha1, image_grads=False)
    assert L == 0.0


def test_alpha_gradient_matches_gpu_central_differences():
    # a nearly fronto-parallel road (row shifts span 0.3 px), so that alpha can
    # sit 0.1 px from every kink of the linear warp
    w = synth.small(256, 160, D=32, ncc_r=3, agg_r=5, seed=23, alpha1=0.002)
    left, right, _ = synth.make_pair(w.scene)
    H = left.shape[0]
    dstar = np.full(left.shape, int(w.delta), np.int16)
    h0 = 1e-2
    h1 = h0 / (H - 1)
    a1 = w.scene.alpha1 + 0.0001
    a0 = kink_free_alpha(w.scene.alpha0 + 0.29, a1, w.delta, H, h0, h1)
    _, da = _gpu_grad(w, left, right, dstar, a0, a1, image_grads=False)
    f = lambda x0, x1: _gpu_grad(w, left, right, dstar, x0, x1, image_grads=False)[0]
    fd0 = (f(a0 + h0, a1) - f(a0 - h0, a1)) / (2 * h0)
    fd1 = (f(a0, a1 + h1) - f(a0, a1 - h1)) / (2 * h1)
    assert da[0] == pytest.approx(fd0, rel=1e-3)
    assert da[1] == pytest.approx(fd1, rel=1e-3)


def test_grad_is_deterministic_in_L_and_alpha():
    w = synth.C1
    left, right, _ = synth.make_pair(w.scene)
    dstar = np.full(left.shape, int(w.delta), np.int16)
    r1 = _gpu_grad(w, left, right, dstar, w.scene.alpha0 + 0.2, w.scene.alpha1)
    r2 = _gpu_grad(w, left, right, dstar, w.scene.alpha0 + 0.2, w.scene.alpha1)
    assert r1[0] == r2[0]
    assert np.array_equal(r1[1], r2[1])


def test_grad_bad_arguments():
    import torch
    from paper_1807_07433_gb300 import sr
    with sr.Matcher(32, 16, 16, 2, 2, 3.0, 10.0) as m:
        img = torch.zeros((16, 32), dtype=torch.uint8, device="cuda")
        ds = torch.zeros((16, 32), dtype=torch.int16, device="cuda")
        with pytest.raises(sr.SrError) as e:
            sr.sr_grad_plane(m.ctx, img, None, 32, ds)
        assert e.value.status == sr.SR_ERR_INVALID_ARG
        with pytest.raises(sr.SrError) as e:
            sr.sr_grad_plane(m.ctx, img, img, 31, ds)
        assert e.value.status == sr.SR_ERR_INVALID_ARG


@pytest.mark.parametrize("method", ["lbfgs", "adam"])
def test_refinement_recovers_the_plane(method):
    """At most 50 evaluations of the CUDA adjoint from a perturbed plane (no
    potholes, so the scene's own plane is where L peaks, up to noise)."""
    import torch
    from paper_1807_07433_gb300 import refine, sr
    sc = synth.Scene(320, 240, 24.0, 0.04, 0, False, 31)
    w = synth.Workload("refine 320x240", sc, D=32, ncc_r=3, agg_r=5, gamma_d=3.0, gamma_r=10.0,
                       delta=12.0)
    left, right, _ = synth.make_pair(sc)
    rng = np.random.default_rng(5)
    a_init = (sc.alpha0 + rng.uniform(-1.5, 1.5), sc.alpha1 + rng.uniform(-0.01, 0.01))
    with sr.Matcher(sc.W, sc.H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r,
                    stream=torch.cuda.current_stream()) as m:
        dstar = torch.full((sc.H, sc.W), int(w.delta), dtype=torch.int16, device="cuda")
        ev = refine.MatcherEvaluator(m, torch.from_numpy(left).cuda(),
                                     torch.from_numpy(right).cuda(), dstar, w.delta)
        res = refine.refine_plane(ev, a_init, sc.H, max_evals=50, method=method)
        L_true = ev.value_and_grad(sc.alpha0, sc.alpha1)[0]
        L_final = ev.value_and_grad(*res.alpha)[0]
    tol = 0.1 if method == "lbfgs" else 0.15   # L peaks within noise (~0.1 px) of the scene plane
    assert abs(res.alpha[0] - sc.alpha0) < tol
    assert abs(res.alpha[1] - sc.alpha1) * (sc.H - 1) < tol
    assert L_final >= L_true - 1e-4 * abs(L_true)


def test_grad_in_16bit_context_uses_fp32_costs():
    """A context that stores FP16 volumes still differentiates the FP32 costs:
    L and dL/dalpha equal those of an FP32 context bit for bit."""
    import torch
    from paper_1807_07433_gb300 import sr
    w = synth.small(120, 70, D=32, ncc_r=3, agg_r=4, seed=24)
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    dl, dr = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    ds = torch.full((H, W), int(w.delta), dtype=torch.int16, device="cuda")
    res = []
    for vt in (sr.SR_VOL_F32, sr.SR_VOL_F16):
        with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, vol_dtype=vt) as m:
            m.set_plane(w.scene.alpha0 + 0.2, w.scene.alpha1, w.delta)
            res.append(m.grad_plane(dl, dr, ds))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])


def test_match_after_grad_is_unchanged():
    """sr_grad_plane uses the context's scratch; a later sr_match is unaffected."""
    import torch
    from helpers import run_gpu
    from paper_1807_07433_gb300 import sr
    w = synth.C1
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    ref = run_gpu(w, left, right)["dfull"]
    dl, dr = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh) as m:
        m.set_plane(w.scene.alpha0 + 0.5, w.scene.alpha1, w.delta)
        m.grad_plane(dl, dr, torch.full((H, W), int(w.delta), dtype=torch.int16, device="cuda"))
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        got = m.match(dl, dr).cpu().numpy()
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.array_equal(got[~np.isnan(got)], ref[~np.isnan(ref)])


def test_full_size_crop_matches_oracle():
    """1280x720 D64 NCC 7x7 bilateral 11x11 scene, the adjoint restricted to
    the crop rows 560-679, cols 560-719 (low in the frame, where alpha1
    matters), at the true plane perturbed by (U[-1.5, 1.5], U[-0.01, 0.01])
    with seed 5: L, dL/dalpha and the image gradients against the oracle,
    which evaluates only the pixels of the set."""
    w = synth.C2
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    dstar = np.full((H, W), -1, np.int16)
    dstar[560:680, 560:720] = int(w.delta)
    rng = np.random.default_rng(5)
    a0 = w.scene.alpha0 + rng.uniform(-1.5, 1.5)
    a1 = w.scene.alpha1 + rng.uniform(-0.01, 0.01)
    _check(w, left, right, dstar, a0, a1)


def test_full_size_crop_gradient_matches_oracle_central_differences():
    """dL/dalpha of the GPU adjoint on the 1280x720 crop (rows 560-679, cols
    560-719) against central differences with step 1e-3 of the FP64 oracle's
    objective.  alpha0 starts at the perturbed plane (seed 5) and moves to
    where no row shift of the rows the crop reads lies within 1.5 steps of an
    integer, so that no difference crosses a kink of the linear warp."""
    import oracle
    w = synth.C2
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    dstar = np.full((H, W), -1, np.int16)
    dstar[560:680, 560:720] = int(w.delta)
    rng = np.random.default_rng(5)
    a0 = w.scene.alpha0 + rng.uniform(-1.5, 1.5)
    a1 = w.scene.alpha1 + rng.uniform(-0.01, 0.01)
    reach = w.agg_r + w.ncc_r
    v = np.arange(560 - reach, 680 + reach, dtype=np.float64)
    h0 = 1e-3
    h1 = h0 / v.max()
    for _ in range(2000):
        s = a0 + a1 * v - w.delta
        frac = s - np.floor(s)
        if np.minimum(frac, 1.0 - frac).min() > 1.5 * h0:
            break
        a0 += 0.0071
    else:
        raise AssertionError("no alpha0 clear of the warp kinks")
    _, da = _gpu_grad(w, left, right, dstar, a0, a1, image_grads=False)
    ds32 = dstar.astype(np.int32)

    def objective(x0, x1):
        p = oracle_params(w)
        p.alpha0, p.alpha1 = x0, x1
        return oracle.objective(p, left.astype(np.float64), right.astype(np.float64), ds32)

    fd0 = (objective(a0 + h0, a1) - objective(a0 - h0, a1)) / (2 * h0)
    fd1 = (objective(a0, a1 + h1) - objective(a0, a1 - h1)) / (2 * h1)
    assert da[0] == pytest.approx(fd0, rel=1e-3)
    assert da[1] == pytest.approx(fd1, rel=1e-3)
