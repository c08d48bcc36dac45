"""GPU road-plane fitting (sr_fit_alpha, sr_fit_roll; Sec. II-A) against the
oracle on the same disparity maps.  The oracle decides inliers by the
definition |d - (a0 + a1 v)| <= tau in double precision; the GPU decides in
single precision (the model rounded to float, one fused multiply-add).  The
two may therefore differ only at pixels whose double-precision residual lies
within the float evaluation's rounding bound of tau ("borderline" pixels):
inlier counts must agree up to each hypothesis' borderline pixels, whose
number is reported; the winning hypothesis and the least-squares line (FP64
sums in different orders: relative 1e-10) must agree wherever the borderline
pixels cannot change them.  The roll fit uses no threshold and is compared
at 1e-10."""
import numpy as np
import pytest

import oracle
from paper_1807_07433_gb300 import synth

pytestmark = pytest.mark.gpu

TAU = 0.5


def _pairs(H, W, n, seed):
    return np.random.default_rng(seed).integers(0, H * W, size=(n, 2)).astype(np.int32)


def _matcher(W, H, w=None):
    import torch
    from paper_1807_07433_gb300 import sr
    w = w or synth.C2
    return sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                      stream=torch.cuda.current_stream())


U32 = 2.0 ** -24


def _borderline(disp_np, pairs):
    """Per hypothesis (None without a model): the pixels whose FP64 residual
    |d - (a0 + a1 v)| is within the single-precision evaluation's rounding
    bound of TAU, 4u (|a0| + |a1| v + |d|); the FP64 line (a0, a1)."""
    H, W = disp_np.shape
    flat = disp_np.ravel().astype(np.float64)
    vv = np.repeat(np.arange(H), W).astype(np.float64)
    out = []
    for i1, i2 in pairs:
        if not (0 <= i1 < H * W and 0 <= i2 < H * W) or i1 // W == i2 // W or \
                np.isnan(flat[i1]) or np.isnan(flat[i2]):
            out.append(None)
            continue
        a1 = (flat[i2] - flat[i1]) / float(i2 // W - i1 // W)
        a0 = flat[i1] - a1 * float(i1 // W)
        res = np.abs(flat - (a0 + a1 * vv))
        eps = 4.0 * U32 * (abs(a0) + abs(a1) * vv + np.abs(flat))
        out.append((np.isfinite(flat) & (np.abs(res - TAU) <= eps), a0, a1))
    return out


def _check_alpha(m, disp_np, pairs):
    import torch
    from paper_1807_07433_gb300 import sr
    got = sr.sr_fit_alpha(m.ctx, torch.from_numpy(disp_np).cuda(), pairs, TAU)
    want = oracle.fit_alpha(disp_np, pairs, TAU)
    border = _borderline(disp_np, pairs)
    nb = np.array([-1 if b is None else int(b[0].sum()) for b in border])
    print(f"borderline pixels: {int(nb[nb > 0].sum())} over {int((nb > 0).sum())} of "
          f"{len(pairs)} hypotheses")
    np.testing.assert_array_equal(got["counts"] < 0, want.counts < 0)
    has = want.counts >= 0
    assert np.all(np.abs(got["counts"][has] - want.counts[has]) <= nb[has])
    if got["best"] != want.best:
        # only borderline pixels can reorder hypotheses
        gb, wb = got["best"], want.best
        assert want.counts[gb] + nb[gb] + nb[wb] >= want.counts[wb]
        return got
    b = want.best
    if nb[b] == 0:
        assert got["n_inliers"] == want.n_inliers
        np.testing.assert_allclose(got["alpha"], want.alpha, rtol=1e-10, atol=1e-12)
    else:   # the two inlier sets differ by borderline pixels only
        assert abs(got["n_inliers"] - want.n_inliers) <= nb[b]
        np.testing.assert_allclose(got["alpha"], want.alpha, rtol=0,
                                   atol=2.0 * TAU * nb[b] / max(want.n_inliers, 1) + 1e-9)
    return got


def test_borderline_residuals_on_the_gpu():
    """Pixels a few float ulps either side of the threshold on the line
    through (v=0, d=1) and (v=3, d=2): the GPU's count differs from the
    oracle's by no more than the borderline pixels (here, all but two)."""
    import torch
    from paper_1807_07433_gb300 import sr
    H, W = 64, 9
    d = np.empty((H, W), np.float32)
    for v in range(H):
        x = np.float32(1.0 + v / 3.0 + TAU)
        for k, step in enumerate(range(-4, 5)):
            y = x
            for _ in range(abs(step)):
                y = np.nextafter(y, np.float32(np.inf if step > 0 else -np.inf))
            d[v, k] = y
    d[0, 0], d[3, 0] = 1.0, 2.0
    pairs = np.array([[0, 3 * W]], np.int32)
    with _matcher(W, H) as m:
        got = sr.sr_fit_alpha(m.ctx, torch.from_numpy(d).cuda(), pairs, TAU)
    want = oracle.fit_alpha(d, pairs, TAU)
    nb = int(_borderline(d, pairs)[0][0].sum())
    assert nb >= H * W - 2 - 2 * H
    assert abs(int(got["counts"][0]) - int(want.counts[0])) <= nb


@pytest.fixture(scope="module")
def c2_disp():
    import torch
    w = synth.C2
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    with _matcher(W, H) as m:
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        d = m.match(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda())
        torch.cuda.synchronize()
        return d.cpu().numpy(), (left, right)


def test_alpha_on_the_full_size_map_matches_oracle(c2_disp):
    disp, _ = c2_disp
    H, W = disp.shape
    pairs = _pairs(H, W, 256, 7)
    with _matcher(W, H) as m:
        got = _check_alpha(m, disp, pairs)
    # the road plane of the scene, potholes and grooves rejected as outliers
    assert abs(got["alpha"][0] - 30.0) < 0.05
    assert abs(got["alpha"][1] - 0.08) * (H - 1) < 0.05


def test_alpha_on_synthetic_lines_with_outliers_and_bad_pairs():
    rng = np.random.default_rng(11)
    H, W = 77, 203
    v = np.arange(H, dtype=np.float64)[:, None] * np.ones((1, W))
    d = (17.25 + 0.0613 * v).astype(np.float32)
    out = rng.random((H, W)) < 0.35
    d[out] += rng.uniform(3, 9, size=out.sum()).astype(np.float32)
    d[rng.random((H, W)) < 0.05] = np.nan
    pairs = _pairs(H, W, 300, 12)
    pairs[:3] = [[4 * W + 1, 4 * W + 7], [-1, 5], [H * W, 0]]     # one row, out of range
    with _matcher(W, H) as m:
        got = _check_alpha(m, d, pairs)
    assert (got["counts"][:3] == -1).all()


def test_roll_matches_oracle(c2_disp):
    import torch
    from paper_1807_07433_gb300 import sr
    disp, _ = c2_disp
    H, W = disp.shape
    patch = (320, 560, 960, 720)                     # near field: the bottom rows
    with _matcher(W, H) as m:
        g, roll, n = sr.sr_fit_roll(m.ctx, torch.from_numpy(disp).cuda(), *patch)
    go, rollo, no = oracle.fit_roll(disp, patch)
    assert n == no
    np.testing.assert_allclose(g, go, rtol=1e-10, atol=1e-12)
    assert roll == pytest.approx(rollo, abs=1e-12)
    assert abs(roll) < 0.02                          # the scene has no roll


def test_roll_of_a_tilted_plane():
    import torch
    from paper_1807_07433_gb300 import sr
    H, W = 90, 160
    u = np.arange(W)[None, :] * np.ones((H, 1))
    v = np.arange(H)[:, None] * np.ones((1, W))
    d = (9.5 - 0.0125 * u + 0.071 * v).astype(np.float32)
    with _matcher(W, H) as m:
        g, roll, n = sr.sr_fit_roll(m.ctx, torch.from_numpy(d).cuda(), -5, 40, 500, 90)
    assert n == 50 * W
    np.testing.assert_allclose(g, [9.5, -0.0125, 0.071], atol=2e-6)
    assert roll == pytest.approx(np.arctan(0.0125 / 0.071), abs=1e-5)


def test_fit_errors():
    import torch
    from paper_1807_07433_gb300 import sr
    H, W = 16, 32
    d = torch.full((H, W), float("nan"), device="cuda")
    with _matcher(W, H) as m:
        with pytest.raises(sr.SrError) as e:
            sr.sr_fit_alpha(m.ctx, d, _pairs(H, W, 8, 1), TAU)
        assert e.value.status == sr.SR_ERR_STATE
        with pytest.raises(sr.SrError) as e:
            sr.sr_fit_roll(m.ctx, d, 10, 10, 10, 20)
        assert e.value.status == sr.SR_ERR_INVALID_ARG
        with pytest.raises(sr.SrError) as e:
            sr.sr_fit_alpha(m.ctx, d, np.zeros((0, 2), np.int32), TAU)
        assert e.value.status == sr.SR_ERR_INVALID_ARG


def test_plane_loop_converges_from_a_perturbed_plane(c2_disp):
    """Match with a wrong plane, fit alpha to the result, match again: the
    full disparity does not depend on the plane used for the transform as
    long as the residuals stay in range, so one fit recovers the plane."""
    import torch
    from paper_1807_07433_gb300 import sr
    _, (left, right) = c2_disp
    w = synth.C2
    H, W = left.shape
    dl, dr = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    a = (w.scene.alpha0 + 1.3, w.scene.alpha1 - 0.004)
    pairs = _pairs(H, W, 256, 9)
    with _matcher(W, H) as m:
        for _ in range(2):
            m.set_plane(a[0], a[1], w.delta)
            disp = m.match(dl, dr)
            a = tuple(sr.sr_fit_alpha(m.ctx, disp, pairs, TAU)["alpha"])
    assert abs(a[0] - 30.0) < 0.05 and abs(a[1] - 0.08) * (H - 1) < 0.05
