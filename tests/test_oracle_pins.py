"""Pins of the FP64 oracle against facts fixed by the paper and mathematics.

Each oracle function is checked against something other than itself, chosen
so that a plausible slip (dropped term, wrong sign or index, transposed
operand, a factor 2 in a Gaussian) fails at least one test:

  warp (Sec. II-A)          integer shifts = np.take with clipping; a linear
                            ramp is shifted exactly; s = 1/2 averages pixels
  block stats (Eqs. 4-5)    numpy mean / population std of edge-padded blocks
  NCC (Eq. 3)               numpy corrcoef of the two blocks; affine
                            invariance c(aI+b) = sign(a) c; +-1 for (anti)
                            identical blocks; 0 for a flat block; |c| <= 1
  volumes (Sec. II-B-1)     index convention against corrcoef; the two-volume
                            identity cost_r(u-d,v,d) = cost_l(u,v,d)
  bilateral (Eqs. 8-10)     scipy gaussian_filter (constant guide, zero-weight
                            border); rho = 0 is the identity; a constant slice
                            stays constant; a two-level guide splits the
                            filter into masked Gaussian filters
  WTA (Sec. II-B-3)         numpy argmax (first index on ties)
  parabola (Eq. 12)         the vertex of a quadratic is recovered exactly
  L-R check (Eq. 11)        hand-built maps
  post-process (Sec. II-C)  integer example of the row shift
  3-D (Sec. II-D)           projecting a known point and reconstructing it
  whole method              exact integer recovery of the residual disparity
                            on noise-free fronto-parallel and tilted planes
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle


def _params(W, H, **kw):
    base = dict(W=W, H=H, D=8, ncc_r=2, agg_r=2, gamma_d=3.0, gamma_r=10.0)
    base.update(kw)
    return oracle.Params(**base)


# ---------------------------------------------------------------- warp (Sec. II-A)

def test_warp_integer_shift_is_clipped_take():
    rng = np.random.default_rng(0)
    W, H = 37, 9
    R = rng.integers(0, 256, (H, W), dtype=np.uint8)
    p = _params(W, H, alpha0=7.0, alpha1=1.0, delta=3.0)  # s(v) = 4 + v, integer
    out = oracle.warp(p, R)
    x = np.arange(W)
    for v in range(H):
        s = 4 + v
        np.testing.assert_array_equal(out[v], R[v, np.clip(x - s, 0, W - 1)].astype(np.float64))


def test_warp_linear_ramp_exact():
    W, H = 100, 6
    x = np.arange(W)
    R = np.tile((2 * x + 10).astype(np.uint8), (H, 1))
    p = _params(W, H, alpha0=3.3, alpha1=0.25, delta=1.0)
    out = oracle.warp(p, R)
    for v in range(H):
        s = 3.3 + 0.25 * v - 1.0
        lo = int(np.ceil(s)) + 1
        hi = W - 1
        xs = x[lo:hi]
        np.testing.assert_allclose(out[v, lo:hi], 2.0 * (xs - s) + 10.0, rtol=0, atol=1e-12)


def test_warp_half_pixel_averages_neighbours():
    rng = np.random.default_rng(1)
    W, H = 20, 3
    R = rng.integers(0, 256, (H, W), dtype=np.uint8)
    p = _params(W, H, alpha0=2.5, alpha1=0.0, delta=0.0)   # s = 2.5 -> k = 2, w = 1/2
    out = oracle.warp(p, R)
    x = np.arange(W)
    want = 0.5 * (R[:, np.clip(x - 2, 0, W - 1)].astype(float) + R[:, np.clip(x - 3, 0, W - 1)])
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-12)


def test_row_shift_and_postprocess():
    p = _params(10, 10, alpha0=30.0, alpha1=0.08, delta=8.0)
    assert oracle.row_shift(p, 100) == pytest.approx(30.0 + 8.0 - 8.0)
    assert oracle.postprocess(p, 7.25, 100) == pytest.approx(7.25 + 30.0)


# ------------------------------------------------------- block stats (Eqs. 4-5)

@pytest.mark.parametrize("r", [1, 2, 3])
def test_block_stats_match_numpy(r):
    rng = np.random.default_rng(2 + r)
    img = rng.uniform(0, 255, (13, 17))
    for (u, v) in [(0, 0), (16, 12), (5, 7), (-3, 4), (20, 2), (8, -2)]:
        mu, sg, var = oracle.block_stats(img, r, u, v)
        blk = np.pad(img, r + 8, mode="edge")[v + 8:v + 8 + 2 * r + 1, u + 8:u + 8 + 2 * r + 1]
        assert mu == pytest.approx(blk.mean(), rel=1e-13)
        assert sg == pytest.approx(blk.std(ddof=0), rel=1e-9, abs=1e-9)
        assert var == pytest.approx(blk.var(ddof=0), rel=1e-9, abs=1e-9)


# ---------------------------------------------------------------- NCC (Eq. 3)

def test_ncc_equals_pearson_corrcoef():
    rng = np.random.default_rng(4)
    L = rng.uniform(0, 255, (15, 30))
    R = rng.uniform(0, 255, (15, 30))
    for r in (1, 2, 3):
        for (ul, ur, v) in [(10, 7, 7), (3, 0, 1), (29, 25, 14), (0, -4, 0), (28, 33, 9)]:
            big_l = np.pad(L, 20, mode="edge")
            big_r = np.pad(R, 20, mode="edge")
            a = big_l[v + 20 - r:v + 21 + r, ul + 20 - r:ul + 21 + r].ravel()
            b = big_r[v + 20 - r:v + 21 + r, ur + 20 - r:ur + 21 + r].ravel()
            want = np.corrcoef(a, b)[0, 1]
            assert oracle.ncc(L, R, r, ul, ur, v) == pytest.approx(want, abs=1e-12)


def test_ncc_affine_invariance():
    rng = np.random.default_rng(5)
    L = rng.uniform(0, 255, (12, 20))
    R = rng.uniform(0, 255, (12, 20))
    for (a, b) in [(2.5, -40.0), (0.3, 100.0), (-1.7, 12.0)]:
        for (ul, ur, v) in [(8, 5, 6), (2, 2, 0), (19, 15, 11)]:
            c0 = oracle.ncc(L, R, 2, ul, ur, v)
            assert oracle.ncc(a * L + b, R, 2, ul, ur, v) == pytest.approx(np.sign(a) * c0, abs=1e-12)
            assert oracle.ncc(L, a * R + b, 2, ul, ur, v) == pytest.approx(np.sign(a) * c0, abs=1e-12)


def test_ncc_identical_and_flat_blocks():
    rng = np.random.default_rng(6)
    L = rng.uniform(0, 255, (12, 20))
    assert oracle.ncc(L, L, 2, 9, 9, 5) == pytest.approx(1.0, abs=1e-13)
    assert oracle.ncc(L, 255.0 - L, 2, 9, 9, 5) == pytest.approx(-1.0, abs=1e-13)
    flat = np.full((12, 20), 77.0)
    assert oracle.ncc(L, flat, 2, 9, 9, 5) == 0.0
    assert oracle.ncc(flat, L, 2, 9, 9, 5) == 0.0
    vals = [oracle.ncc(L, rng.uniform(0, 255, (12, 20)), 2, u, u - 1, 4) for u in range(1, 19)]
    assert max(abs(c) for c in vals) <= 1.0 + 1e-12


# --------------------------------------------------- volumes (Sec. II-B-1)

def test_volume_index_convention_and_two_volume_identity():
    rng = np.random.default_rng(7)
    W, H, D = 26, 11, 6
    L = rng.integers(0, 256, (H, W), dtype=np.uint8)
    R = rng.integers(0, 256, (H, W), dtype=np.uint8)
    p = _params(W, H, D=D, ncc_r=2, agg_r=1, alpha0=2.0, alpha1=0.1, delta=1.0)
    res = oracle.match(p, L, R, want=("warped", "cost_l", "cost_r"))
    Rw = res.warped
    np.testing.assert_allclose(Rw, oracle.warp(p, R), atol=0)
    # reference volume: left block u against warped-target block u-d
    for (u, v, d) in [(10, 5, 3), (0, 0, 0), (25, 10, 5), (3, 4, 5), (17, 2, 1)]:
        big_l = np.pad(L.astype(float), 12, mode="edge")
        big_r = np.pad(Rw, 12, mode="edge")
        a = big_l[v + 10:v + 15, u + 10:u + 15].ravel()
        b = big_r[v + 10:v + 15, u - d + 10:u - d + 15].ravel()
        assert res.cost_l[v, u, d] == pytest.approx(np.corrcoef(a, b)[0, 1], abs=1e-12)
    # Sec. II-B-1: c at (u,v,d) of the reference volume equals c at (u-d,v,d) of the target one
    for d in range(D):
        np.testing.assert_allclose(res.cost_r[:, :W - d, d], res.cost_l[:, d:, d], rtol=0, atol=1e-15)


# ---------------------------------------------------- bilateral (Eqs. 8-10)

def _gauss_norm(slice_, mask, gamma_d, rho):
    sig = gamma_d / np.sqrt(2.0)           # exp(-r^2/gamma^2) = exp(-r^2/(2 sig^2))
    kw = dict(sigma=sig, mode="constant", cval=0.0, truncate=rho / sig)
    num = ndimage.gaussian_filter(slice_ * mask, **kw)
    den = ndimage.gaussian_filter(mask.astype(float), **kw)
    return num, den


@pytest.mark.parametrize("rho,gamma_d", [(2, 1.5), (4, 3.0), (5, 4.0)])
def test_bilateral_constant_guide_is_normalised_gaussian(rho, gamma_d):
    rng = np.random.default_rng(8)
    H, W = 19, 23
    s = rng.uniform(-1, 1, (H, W))
    g = np.full((H, W), 50.0)
    out = oracle.bilateral_slice(s, g, rho, gamma_d, 10.0)
    num, den = _gauss_norm(s, np.ones((H, W)), gamma_d, rho)
    np.testing.assert_allclose(out, num / den, rtol=0, atol=1e-12)


def test_bilateral_identity_and_constant():
    rng = np.random.default_rng(9)
    s = rng.uniform(-1, 1, (9, 14))
    g = rng.uniform(0, 255, (9, 14))
    np.testing.assert_allclose(oracle.bilateral_slice(s, g, 0, 3.0, 10.0), s, atol=1e-15)
    c = np.full((9, 14), 0.37)
    np.testing.assert_allclose(oracle.bilateral_slice(c, g, 3, 3.0, 10.0), c, atol=1e-14)


def test_bilateral_two_level_guide_splits_into_masked_gaussians():
    rng = np.random.default_rng(10)
    H, W, rho, gd, gr = 16, 24, 3, 2.0, 30.0
    s = rng.uniform(-1, 1, (H, W))
    A = np.zeros((H, W), bool)
    A[:, :11] = True
    A[3:7, 15:20] = True
    B = ~A
    g = np.where(A, 100.0, 100.0 + gr)     # cross-level intensity weight is exp(-1)
    out = oracle.bilateral_slice(s, g, rho, gd, gr)
    nA, dA = _gauss_norm(s, A, gd, rho)
    nB, dB = _gauss_norm(s, B, gd, rho)
    e = np.exp(-1.0)
    want = np.where(A, (nA + e * nB) / (dA + e * dB), (nB + e * nA) / (dB + e * dA))
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-12)


# -------------------------------------------------- WTA, parabola, L-R, 3-D

def test_wta_is_first_argmax():
    rng = np.random.default_rng(11)
    for _ in range(200):
        c = np.round(rng.uniform(-1, 1, rng.integers(1, 70)), 1)   # many exact ties
        best, gap = oracle.wta(c)
        assert best == int(np.argmax(c))
        if c.size > 1:
            assert gap == pytest.approx(c[best] - np.sort(np.delete(c, best))[-1])


def test_parabola_recovers_quadratic_vertex():
    rng = np.random.default_rng(12)
    D = 32
    d = np.arange(D, dtype=float)
    for _ in range(100):
        d0 = rng.uniform(1.0, D - 2.0)
        a, b = rng.uniform(0.01, 2.0), rng.uniform(-1, 1)
        c = -a * (d - d0) ** 2 + b
        best, _ = oracle.wta(c)
        ds, den = oracle.parabola(c, best)
        assert best == int(np.rint(d0)) or abs(d0 - np.floor(d0) - 0.5) < 1e-9
        assert ds == pytest.approx(d0, abs=1e-9)
        assert den == pytest.approx(-4.0 * a, rel=1e-9)
    c = -(d - 0.2) ** 2
    assert oracle.parabola(c, 0) == (0.0, 0.0)
    c = -(d - D + 1.1) ** 2
    assert oracle.parabola(c, D - 1) == (float(D - 1), 0.0)


def test_lr_check_hand_built():
    ltar = np.array([0, 1, 2, 3, 4, 5, 6, 7], np.int32)
    assert oracle.lr_valid(5, 2, ltar, 1.0)        # target at 3 has 3: |2-3| = 1
    assert not oracle.lr_valid(6, 2, ltar, 1.0)    # target at 4 has 4: |2-4| = 2
    assert oracle.lr_valid(6, 2, ltar, 2.0)
    assert not oracle.lr_valid(1, 2, ltar, 1.0)    # match falls off the image
    assert oracle.lr_valid(2, 2, np.array([2, 9, 9], np.int32), 0.0)
    assert not oracle.lr_valid(2, 2, np.array([1, 9, 9], np.int32), 0.0)


def test_reconstruct_inverts_projection():
    p = _params(1280, 720, f_px=700.0, baseline=120.0)
    u0, v0 = (1280 - 1) / 2, (720 - 1) / 2
    rng = np.random.default_rng(13)
    for _ in range(20):
        X, Y, Z = rng.uniform(-2000, 2000), rng.uniform(500, 1500), rng.uniform(1500, 8000)
        u = int(round(700.0 * X / Z + u0))
        v = int(round(700.0 * Y / Z + v0))
        Xs, Ys = (u - u0) * Z / 700.0, (v - v0) * Z / 700.0      # point on the pixel's ray
        d = 700.0 * 120.0 / Z
        got = oracle.reconstruct(p, d, u, v)
        np.testing.assert_allclose(got, (Xs, Ys, Z), rtol=1e-12)
    assert all(np.isnan(oracle.reconstruct(p, 0.0, 3, 3)))
    assert all(np.isnan(oracle.reconstruct(p, float("nan"), 3, 3)))


# ------------------------------------------------------------ whole method

def _textured(rng, H, W):
    t = ndimage.gaussian_filter(rng.uniform(0, 255, (H, W)), 1.0)
    t = (t - t.mean()) / t.std() * 45 + 128
    return t


def test_fronto_parallel_plane_exact_integer_recovery():
    rng = np.random.default_rng(14)
    H, W, D, delta, a0 = 40, 96, 12, 4.0, 11.0
    tex = np.clip(np.rint(_textured(rng, H, W + 40)), 0, 255).astype(np.uint8)
    L = tex[:, :W]
    R = tex[:, int(a0):int(a0) + W]               # right(x) = left(x + a0): disparity a0
    p = _params(W, H, D=D, ncc_r=2, agg_r=3, alpha0=a0, alpha1=0.0, delta=delta)
    res = oracle.match(p, L, R, want=("lbl_l", "lbl_r", "valid", "dfull"))
    m = p.ncc_r + p.agg_r + 1
    inner = (slice(m, H - m), slice(m + D, W - m - D))
    assert np.all(res.lbl_l[inner] == int(delta))
    assert np.all(res.lbl_r[inner] == int(delta))
    assert np.all(res.valid[inner] == 1)
    np.testing.assert_allclose(res.dfull[inner], a0, atol=0.5)


def test_tilted_plane_recovery_with_true_plane():
    rng = np.random.default_rng(15)
    H, W, D, delta = 60, 120, 12, 5.0
    a0, a1 = 9.3, 0.07
    texf = _textured(rng, H, W + 60)
    xs = np.arange(W + 60, dtype=float)
    L = np.clip(np.rint(texf[:, :W]), 0, 255).astype(np.uint8)
    Rf = np.empty((H, W))
    for v in range(H):
        Rf[v] = np.interp(np.arange(W) + a0 + a1 * v, xs, texf[v])   # right(x) = left(x + d(v))
    R = np.clip(np.rint(Rf), 0, 255).astype(np.uint8)
    p = _params(W, H, D=D, ncc_r=2, agg_r=3, alpha0=a0, alpha1=a1, delta=delta)
    res = oracle.match(p, L, R, want=("lbl_l", "dfull"))
    m = p.ncc_r + p.agg_r + 1
    inner = (slice(m, H - m), slice(m + D, W - m - D))
    assert np.mean(res.lbl_l[inner] == int(delta)) >= 0.99
    true_d = (a0 + a1 * np.arange(H))[:, None] * np.ones((1, W))
    err = np.abs(res.dfull[inner] - true_d[inner])
    assert np.nanmedian(err) < 0.1


def test_pixel_sampler_agrees_with_full_frame():
    from paper_1807_07433_gb300 import synth
    w = synth.small(48, 30, D=8, ncc_r=1, agg_r=2, seed=3)
    L, R, _ = synth.make_pair(w.scene)
    p = oracle.Params(W=48, H=30, D=8, ncc_r=1, agg_r=2, gamma_d=w.gamma_d, gamma_r=w.gamma_r,
                      alpha0=w.scene.alpha0, alpha1=w.scene.alpha1, delta=w.delta)
    full = oracle.match(p, L, R)
    rng = np.random.default_rng(0)
    us = rng.integers(0, 48, 60)
    vs = rng.integers(0, 30, 60)
    smp = oracle.match_pixels(p, L, R, us, vs)
    np.testing.assert_array_equal(smp["lbl_l"], full.lbl_l[vs, us])
    np.testing.assert_allclose(smp["dsub"], full.dsub[vs, us], atol=1e-12)
    np.testing.assert_array_equal(smp["valid"], full.valid[vs, us])
    np.testing.assert_allclose(smp["dfull"], full.dfull[vs, us], atol=1e-12)
