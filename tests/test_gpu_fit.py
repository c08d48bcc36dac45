"""GPU road-plane fitting (sr_fit_alpha, sr_fit_roll; Sec. II-A) against the
oracle on the same disparity maps: inlier counts, the winning hypothesis and
the pixel count are integers and must match exactly (both sides decide in
single precision with one fused multiply-add); the least-squares results are
FP64 sums in different orders (relative 1e-10)."""
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


def _check_alpha(m, disp_np, pairs):
    import torch
    from paper_1807_07433_gb300 import sr
    got = sr.sr_fit_alpha(m.ctx, torch.from_numpy(disp_np).cuda(), pairs, TAU)
    want = oracle.fit_alpha(disp_np, pairs, TAU)
    np.testing.assert_array_equal(got["counts"], want.counts)
    assert got["best"] == want.best and got["n_inliers"] == want.n_inliers
    np.testing.assert_allclose(got["alpha"], want.alpha, rtol=1e-10, atol=1e-12)
    return got


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
