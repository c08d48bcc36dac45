"""Shared helpers for the parity tests: run the CUDA path through the C ABI and
the FP64 oracle on the same seeded inputs, and compare them with the stated
tolerances.

Tolerances (derivation in the design notes; FP32 unit roundoff u = 2^-24):
  TOL_WARP   1e-4  warped intensities (<= 255, two FP32 ops: ~3e-5)
  TOL_MU     1e-4  block means (<= 255, n <= 121 FP32 adds)
  TOL_SIG    1e-5  relative error of 1/(n sigma)
  TOL_COST   1e-4  NCC cost in [-1, 1] (centred FP32 dot product; the bound
                   grows like n*u*sum|a||s|/(n sigma_f sigma_s), largest on
                   near-flat blocks)
  TOL_AGG    2e-5  aggregated cost (weighted mean of costs, FP32 weights)
  TAU_TIE    1e-4  a WTA label may differ only where the oracle's best and
                   second-best aggregated costs are closer than this
  TOL_DSUB   1e-3  px, subpixel disparity away from near-ties: where labels
                   agree, the oracle's top-2 gap is >= TAU_TIE and its parabola
                   denominator |den| >= DEN_MIN.  The Eq. 12 offset moves by
                   about 6 eps / |den| for a cost error eps; FP32 storage of
                   the warped image alone gives eps ~ 1e-6 on low-texture
                   blocks, so |den| < 6e-3 is an ill-conditioned (near-tie)
                   parabola.
  DEN_MIN    6e-3
  AGREE_MIN  0.999 fraction of integer disparities that must agree
"""
from __future__ import annotations

import numpy as np

TOL_WARP = 1e-4
TOL_MU = 1e-4
TOL_SIG = 1e-5
TOL_COST = 1e-4
TOL_AGG = 2e-5
TAU_TIE = 1e-4
TOL_DSUB = 1e-3
DEN_MIN = 6e-3
AGREE_MIN = 0.999


def oracle_params(w):
    import oracle
    return oracle.Params(W=w.scene.W, H=w.scene.H, D=w.D, ncc_r=w.ncc_r, agg_r=w.agg_r,
                         gamma_d=w.gamma_d, gamma_r=w.gamma_r, lr_thresh=w.lr_thresh,
                         alpha0=w.scene.alpha0, alpha1=w.scene.alpha1, delta=w.delta,
                         f_px=w.f_px, baseline=w.baseline_mm)


def run_gpu(w, left, right, keep_agg=False, buffers=(), vol_dtype=0):
    """Run sr_match (+ sr_reconstruct) on cuda:0 through the C ABI; return numpy arrays."""
    import torch
    from paper_1807_07433_gb300 import sr
    H, W = left.shape
    dl = torch.from_numpy(left).cuda()
    dr = torch.from_numpy(right).cuda()
    out = {}
    with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                    vol_dtype=vol_dtype, stream=torch.cuda.current_stream()) as m:
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        m.set_camera(w.f_px, w.baseline_mm)
        if keep_agg:
            sr.sr_set_debug(m.ctx, sr.SR_DEBUG_KEEP_AGG)
        wta = torch.empty((H, W), dtype=torch.int16, device="cuda")
        disp = m.match(dl, dr, wta=wta)
        xyz = m.reconstruct(disp)
        torch.cuda.synchronize()
        out["dfull"] = disp.cpu().numpy()
        out["wta"] = wta.cpu().numpy()
        out["xyz"] = xyz.cpu().numpy()
        for name, which in buffers:
            out[name] = m.buffer(which)
    return out


def run_oracle(w, left, right, want):
    import oracle
    return oracle.match(oracle_params(w), left, right, want=want)


def label_report(gpu_lbl, orc_lbl, orc_gap):
    """Return (agree fraction, mismatches that are not near-ties)."""
    diff = gpu_lbl.astype(np.int64) != orc_lbl.astype(np.int64)
    bad = diff & ~(orc_gap < TAU_TIE)
    return 1.0 - diff.mean(), int(bad.sum())


def kink_free_alpha(a0, a1, delta, H, h0, h1, step=0.0071):
    """alpha0 near a0 such that every row shift s(v) = alpha0 + alpha1 v - delta
    (Sec. II-A) stays more than ten steps from an integer, where the linear
    warp has a kink; a step h1 in alpha1 moves row v by h1 * v."""
    v = np.arange(H)
    for _ in range(400):
        s = a0 + a1 * v - delta
        frac = s - np.floor(s)
        if np.minimum(frac, 1.0 - frac).min() > 10.0 * max(h0, h1 * (H - 1)):
            return a0
        a0 += step
    raise AssertionError("no kink-free alpha0 found")


def near_flat_slack(warped, D, ncc_r, agg_r, e=TOL_WARP):
    """Extra error allowed where a warped-target block is nearly flat.

    A cost of Eq. 3 is a centred dot product over n sigma_l sigma_r.  An
    intensity error e in the warped block (at most TOL_WARP, the bound
    asserted on the warped image; a test may pass the error it measured)
    moves the numerator by at most sqrt(n) sigma_l sqrt(n) e
    (Cauchy-Schwarz) and sigma_r by at most e, so the cost moves by at most
    2 e / sigma_r: large where sigma_r is small but above the flat
    threshold.  Returns (slack_l, slack_r) of shape [H][W][D] for the two
    cost volumes and their aggregates (the maximum over the bilateral
    window, since a weighted mean moves by no more than its largest term).
    A block whose variance lies within 20 % of the flat threshold may be
    classed differently by the two sides; there the slack is 2 (any cost)."""
    from scipy.ndimage import maximum_filter
    H, W = warped.shape
    r = ncc_r
    # block sigma of the warped image at centres x in [-(D-1), W), clamp-to-edge
    pad = np.pad(warped, ((r, r), (D - 1 + r, r)), mode="edge")
    n = (2 * r + 1) ** 2
    s = np.zeros((H, W + D - 1))
    s2 = np.zeros((H, W + D - 1))
    for j in range(2 * r + 1):
        for i in range(2 * r + 1):
            blk = pad[j:j + H, i:i + W + D - 1]
            s += blk
            s2 += blk * blk
    var = np.maximum(s2 / n - (s / n) ** 2, 0.0)
    slack = np.where(var > 0, 2.0 * e / np.sqrt(np.maximum(var, 1e-300)), 0.0)
    slack = np.where(var < 0.8e-6, 0.0, slack)                 # flat on both sides: c = 0
    slack = np.where(np.abs(var - 1e-6) <= 0.2e-6, 2.0, slack)  # flatness may flip
    slack = np.minimum(slack, 2.0)
    u = np.arange(W)[None, :, None]
    d = np.arange(D)[None, None, :]
    # cost_l(u, d) pairs the left block at u with the warped block at u - d;
    # cost_r(u, d) pairs the left block at u + d with the warped block at u
    sl = slack[:, (u - d + D - 1)[0]]
    sr = np.broadcast_to(slack[:, D - 1:][:, :, None], (H, W, D))
    k = 2 * agg_r + 1
    agg_l = maximum_filter(sl, size=(k, k, 1), mode="nearest")
    agg_r = maximum_filter(sr, size=(k, k, 1), mode="nearest")
    return sl, sr, agg_l, agg_r
