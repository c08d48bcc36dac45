"""GPU restricted search (sr_match_restricted) against the oracle's
orc_match_restricted, plus exact identities: the band kernel (16-disparity
slices through a TMA tensor map) equals the full-D kernel with windowed WTA
bit for bit, and a radius of D-1 equals sr_match away from near-ties."""
import numpy as np
import pytest

import oracle
from helpers import AGREE_MIN, DEN_MIN, TAU_TIE, TOL_DSUB, label_report, oracle_params
from paper_1807_07433_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(w, left, right, centre, radius, vt=0, no_band=False):
    import torch
    from paper_1807_07433_gb300 import sr
    H, W = left.shape
    with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                    vol_dtype=vt, stream=torch.cuda.current_stream()) as m:
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        if no_band:
            sr.sr_set_debug(m.ctx, sr.SR_DEBUG_NO_BAND)
        wta = torch.empty((H, W), dtype=torch.int16, device="cuda")
        c = None if centre is None else torch.from_numpy(centre.astype(np.int16)).cuda()
        disp = m.match_restricted(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(),
                                  radius, centre=c, wta=wta)
        torch.cuda.synchronize()
        return {"dfull": disp.cpu().numpy(), "wta": wta.cpu().numpy(),
                "lbl_r": m.buffer(sr.SR_BUF_WTA_R), "dsub": m.buffer(sr.SR_BUF_DSUB)}


def _centres(w, left, right, kind, seed=0):
    H, W = left.shape
    if kind == "plane":
        return None
    rng = np.random.default_rng(seed)
    if kind == "labels":        # a previous frame: the full search's labels, jittered
        full = oracle.match(oracle_params(w), left, right, want=("lbl_l",))
        return np.clip(full.lbl_l + rng.integers(-1, 2, size=(H, W)), 0, w.D - 1)
    return rng.integers(0, w.D, size=(H, W))      # "random": most tiles need all D


CASES = [
    (synth.small(203, 77, D=64, ncc_r=3, agg_r=5, seed=31), "plane", 4),
    (synth.small(203, 77, D=64, ncc_r=3, agg_r=5, seed=31), "labels", 3),
    (synth.small(150, 61, D=32, ncc_r=2, agg_r=4, seed=32), "labels", 2),
    (synth.small(150, 61, D=32, ncc_r=2, agg_r=4, seed=32), "random", 5),
    (synth.small(97, 45, D=16, ncc_r=2, agg_r=3, seed=33), "labels", 2),
    (synth.small(70, 38, D=64, ncc_r=1, agg_r=7, seed=34), "plane", 7),
]


@pytest.mark.parametrize("w,kind,radius", CASES, ids=lambda x: getattr(x, "name", str(x)))
def test_restricted_matches_oracle(w, kind, radius):
    left, right, _ = synth.make_pair(w.scene)
    centre = _centres(w, left, right, kind)
    g = _run(w, left, right, centre, radius)
    c = np.full(left.shape, int(round(w.delta))) if centre is None else centre
    o = oracle.match(oracle_params(w), left, right, centre=c, radius=radius,
                     want=("lbl_l", "lbl_r", "gap_l", "gap_r", "den_l", "dsub", "dfull"))
    agree, bad = label_report(g["wta"], o.lbl_l, o.gap_l)
    assert agree >= AGREE_MIN and bad == 0, (agree, bad)
    agree_r, bad_r = label_report(g["lbl_r"], o.lbl_r, o.gap_r)
    assert agree_r >= AGREE_MIN and bad_r == 0, (agree_r, bad_r)
    ok = (g["wta"] == o.lbl_l) & (o.gap_l >= TAU_TIE) & \
        ((np.abs(o.den_l) >= DEN_MIN) | (o.den_l == 0))
    assert np.abs(g["dsub"][ok] - o.dsub[ok]).max() <= TOL_DSUB


@pytest.mark.parametrize("vt", [0, 1, 2])
@pytest.mark.parametrize("kind", ["plane", "labels"])
def test_band_kernel_equals_full_kernel_bitwise(vt, kind):
    w = synth.small(203, 77, D=64, ncc_r=3, agg_r=5, seed=35)
    left, right, _ = synth.make_pair(w.scene)
    centre = _centres(w, left, right, kind, seed=3)
    a = _run(w, left, right, centre, 4, vt=vt)
    b = _run(w, left, right, centre, 4, vt=vt, no_band=True)
    for k in ("wta", "lbl_r", "dsub"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    np.testing.assert_array_equal(np.isnan(a["dfull"]), np.isnan(b["dfull"]))


def test_radius_d_minus_one_equals_sr_match():
    """A window of radius D-1 is the full search.  The restricted search
    computes its two volumes with the direct NCC kernel (per-tile disparity
    ranges) and sr_match its one extended volume with the exact-sum kernel, so
    their costs agree to rounding: the maps are equal away from the oracle's
    near-ties, and the subpixel disparities within the parity tolerance."""
    import torch
    from paper_1807_07433_gb300 import sr
    w = synth.small(150, 61, D=32, ncc_r=2, agg_r=4, seed=36)
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    dl, dr = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh) as m:
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        wf = torch.empty((H, W), dtype=torch.int16, device="cuda")
        wr = torch.empty((H, W), dtype=torch.int16, device="cuda")
        full = m.match(dl, dr, wta=wf).cpu().numpy()
        rest = m.match_restricted(dl, dr, w.D - 1, wta=wr).cpu().numpy()
        wf, wr = wf.cpu().numpy(), wr.cpu().numpy()
    o = oracle.match(oracle_params(w), left, right, want=("gap_l", "gap_r", "den_l"))
    # the target view's labels decide validity at u - d: a pixel is firm when
    # neither gap it depends on is a near-tie
    firm = o.gap_l >= TAU_TIE
    ur = np.arange(W)[None, :] - np.clip(wf, 0, w.D - 1)
    firm &= np.where(ur >= 0, o.gap_r[np.arange(H)[:, None], np.clip(ur, 0, W - 1)] >= TAU_TIE,
                     True)
    np.testing.assert_array_equal(wf[firm], wr[firm])
    np.testing.assert_array_equal(np.isnan(full)[firm], np.isnan(rest)[firm])
    sub = firm & np.isfinite(full) & (np.abs(o.den_l) >= DEN_MIN)
    assert np.abs(full[sub] - rest[sub]).max(initial=0.0) <= TOL_DSUB
    assert firm.mean() >= 0.95   # the comparison covers most pixels


def test_restricted_bad_arguments():
    import torch
    from paper_1807_07433_gb300 import sr
    with sr.Matcher(64, 32, 32, 2, 2, 3.0, 10.0) as m:
        img = torch.zeros((32, 64), dtype=torch.uint8, device="cuda")
        for r in (-1, 32):
            with pytest.raises(sr.SrError) as e:
                m.match_restricted(img, img, r)
            assert e.value.status == sr.SR_ERR_INVALID_ARG


def test_window_gives_a_smaller_search_range():
    """A search of 0..D'-1 with D' = 24 on a D = 32 context: every centre at
    floor((D'-1)/2) = 11 with radius floor(D'/2) = 12 makes each window
    exactly [0, 23], so the result is the oracle's full search with D = 24."""
    w32 = synth.small(150, 61, D=32, ncc_r=2, agg_r=4, seed=37)
    w24 = synth.small(150, 61, D=24, ncc_r=2, agg_r=4, seed=37)
    left, right, _ = synth.make_pair(w32.scene)
    g = _run(w32, left, right, np.full(left.shape, 11), 12)
    o = oracle.match(oracle_params(w24), left, right,
                     want=("lbl_l", "lbl_r", "gap_l", "gap_r", "den_l", "dsub", "dfull"))
    agree, bad = label_report(g["wta"], o.lbl_l, o.gap_l)
    assert agree >= AGREE_MIN and bad == 0, (agree, bad)
    agree_r, bad_r = label_report(g["lbl_r"], o.lbl_r, o.gap_r)
    assert agree_r >= AGREE_MIN and bad_r == 0, (agree_r, bad_r)
    ok = (g["wta"] == o.lbl_l) & (o.gap_l >= TAU_TIE) & \
        ((np.abs(o.den_l) >= DEN_MIN) | (o.den_l == 0))
    assert np.abs(g["dsub"][ok] - o.dsub[ok]).max() <= TOL_DSUB
    both = ok & np.isfinite(g["dfull"]) & np.isfinite(o.dfull)
    assert both.mean() > 0.5
    assert np.abs(g["dfull"][both] - o.dfull[both]).max() <= TOL_DSUB
