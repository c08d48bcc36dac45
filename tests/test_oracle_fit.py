"""Pins of the oracle's road-plane fitting (Sec. II-A): alpha of Eq. 2 by
least squares with RANSAC over point pairs of a disparity map, and the roll
angle from a plane fitted to a near-field patch.

The inlier test is the definition |d - (a0 + a1 v)| <= tau in double
precision.  Most pins use data without borderline residuals (every pixel is
either on the model up to float rounding or at least 3 px away); one pin
places pixels a float ulp or two either side of the boundary, where a
single-precision evaluation of the same test decides differently, and
checks the oracle against float64 brute force there.  The least-squares
results are checked against numpy.linalg.lstsq on the same inlier set."""
import math

import numpy as np
import pytest

import oracle

TAU = 0.5


def _line_map(H=60, W=80, a0=21.5, a1=0.0731, seed=0, p_out=0.3, p_nan=0.05):
    rng = np.random.default_rng(seed)
    v = np.arange(H, dtype=np.float64)[:, None] * np.ones((1, W))
    d = (a0 + a1 * v).astype(np.float32)
    out = rng.random((H, W)) < p_out
    d[out] += rng.uniform(3.0, 10.0, size=out.sum()).astype(np.float32) * \
        rng.choice([-1, 1], size=out.sum())
    nan = rng.random((H, W)) < p_nan
    d[nan] = np.nan
    return d, ~out & ~nan


def _pairs(H, W, n, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, H * W, size=(n, 2)).astype(np.int32)


def test_counts_equal_brute_force_and_best_is_the_true_line():
    d, inl = _line_map()
    H, W = d.shape
    pairs = _pairs(H, W, 64, 1)
    pairs[0] = (5 * W + 3, 5 * W + 9)            # same row: no model
    pairs[1] = (np.argwhere(np.isnan(d.ravel()))[0, 0], 7)   # an invalid point
    fit = oracle.fit_alpha(d, pairs, TAU)
    assert fit.counts[0] == -1 and fit.counts[1] == -1
    flat = d.ravel().astype(np.float64)
    vv = np.repeat(np.arange(H), W)
    for h, (i1, i2) in enumerate(pairs):
        if fit.counts[h] < 0:
            continue
        a1 = (flat[i2] - flat[i1]) / (vv[i2] - vv[i1])
        a0 = flat[i1] - a1 * vv[i1]
        res = np.abs(flat - (a0 + a1 * vv))
        assert fit.counts[h] == int(np.sum(res <= TAU)), h
    assert fit.n_inliers == inl.sum() == fit.counts[fit.best]
    assert fit.best == int(np.argmax(fit.counts))          # first of the maxima
    # least squares over the best's inliers = numpy lstsq on the true inliers
    A = np.stack([np.ones(inl.sum()), vv.reshape(H, W)[inl]], 1)
    ref = np.linalg.lstsq(A, d[inl].astype(np.float64), rcond=None)[0]
    np.testing.assert_allclose(fit.alpha, ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(fit.alpha, [21.5, 0.0731], rtol=0, atol=2e-6)


def _float_inlier_count(flat, vv, a0, a1, tau):
    """The inlier test evaluated in single precision with one fused
    multiply-add (a1 v + a0 is exact in float64 for float a0, a1 and
    small integer v, so rounding it once to float32 is the fma)."""
    a0f, a1f = np.float32(a0), np.float32(a1)
    m = (np.float64(a1f) * vv + np.float64(a0f)).astype(np.float32)
    r = np.abs(flat.astype(np.float32) - m)
    return int(np.sum(r <= np.float32(tau)))


def test_borderline_residuals_follow_the_double_precision_definition():
    """Pixels within a float ulp or two of |d - (a0 + a1 v)| = tau, on the
    line through (v=0, d=1) and (v=3, d=2) (a1 = 1/3, not a float): the
    oracle's counts equal float64 brute force, and the data is chosen so
    that the single-precision test counts differently."""
    H, W = 64, 9
    d = np.empty((H, W), np.float32)
    vv = np.repeat(np.arange(H), W).astype(np.float64)
    for v in range(H):
        x = np.float32(1.0 + v / 3.0 + TAU)
        for k, step in enumerate(range(-4, 5)):       # x and 4 floats either side
            y = x
            for _ in range(abs(step)):
                y = np.nextafter(y, np.float32(np.inf if step > 0 else -np.inf))
            d[v, k] = y
    d[0, 0], d[3, 0] = 1.0, 2.0                       # the hypothesis' two points
    pairs = np.array([[0, 3 * W]], np.int32)
    fit = oracle.fit_alpha(d, pairs, TAU)
    flat = d.ravel().astype(np.float64)
    a1 = (2.0 - 1.0) / 3.0
    a0 = 1.0 - a1 * 0.0
    want = int(np.sum(np.abs(flat - (a0 + a1 * vv)) <= TAU))
    assert fit.counts[0] == want
    assert _float_inlier_count(flat, vv, a0, a1, TAU) != want
    inl = np.abs(flat - (a0 + a1 * vv)) <= TAU
    A = np.stack([np.ones(inl.sum()), vv[inl]], 1)
    ref = np.linalg.lstsq(A, flat[inl], rcond=None)[0]
    np.testing.assert_allclose(fit.alpha, ref, rtol=1e-12, atol=1e-12)


def test_no_model_at_all():
    d = np.full((10, 12), np.nan, np.float32)
    fit = oracle.fit_alpha(d, _pairs(10, 12, 8, 2), TAU)
    assert fit.best == -1 and (fit.counts == -1).all() and fit.n_inliers == 0


def test_ties_go_to_the_first_hypothesis():
    d, _ = _line_map(p_out=0.0, p_nan=0.0)
    H, W = d.shape
    pairs = np.array([[0, 3 * W], [W, 5 * W + 2], [2 * W + 1, 9 * W]], np.int32)
    fit = oracle.fit_alpha(d, pairs, TAU)
    assert (fit.counts == H * W).all() and fit.best == 0


def test_roll_plane_recovered_and_equals_lstsq():
    H, W = 50, 70
    g_true = (12.25, -0.0213, 0.0842)
    u = np.arange(W)[None, :] * np.ones((H, 1))
    v = np.arange(H)[:, None] * np.ones((1, W))
    d = (g_true[0] + g_true[1] * u + g_true[2] * v).astype(np.float32)
    rng = np.random.default_rng(3)
    d[rng.random((H, W)) < 0.1] = np.nan
    d[:10, :] = 999.0                                 # outside the patch: ignored
    patch = (5, 20, 60, 50)                           # u_lo, v_lo, u_hi, v_hi
    g, roll, n = oracle.fit_roll(d, patch)
    sub = d[20:50, 5:60]
    m = np.isfinite(sub)
    assert n == m.sum()
    A = np.stack([np.ones(m.sum()), u[20:50, 5:60][m], v[20:50, 5:60][m]], 1)
    ref = np.linalg.lstsq(A, sub[m].astype(np.float64), rcond=None)[0]
    np.testing.assert_allclose(g, ref, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(g, g_true, rtol=0, atol=2e-6)
    assert roll == pytest.approx(math.atan(-g[1] / g[2]), rel=1e-15)
    assert roll == pytest.approx(math.atan(0.0213 / 0.0842), abs=1e-4)


def test_roll_singular_patch():
    d = np.full((20, 20), 5.0, np.float32)
    g, roll, n = oracle.fit_roll(d, (3, 4, 10, 5))   # one row: v is constant
    assert n == -1
