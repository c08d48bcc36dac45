"""The accuracy gate on whole frames: the plain FP32 GPU form against the FP64
oracle on every pixel of the 1280x720x64 benchmark frame and of the
1920x1080x64 frame, both with NCC 7x7 and bilateral 11x11.

The gate (Eqs. 3, 8-12 and Sec. II-C on the synthetic road scenes):
  * at least 99.9 % of the integer disparities (reference-view WTA labels,
    Sec. II-B-3) agree with the oracle's;
  * every label that differs is a near-tie: the oracle's best and
    second-best aggregated costs are closer than TAU_TIE;
  * where the labels agree, the pixel is not a near-tie and the oracle's
    parabola (Eq. 12) is well conditioned (|den| >= DEN_MIN), the full
    disparity differs by at most TOL_DSUB px;
  * the L-R check (Eq. 11) gives the oracle's validity wherever both label
    maps agree at the pixel and at its match.
The oracle runs the whole frame on the host cores (about 1.4 s for the
1280x720 frame on 16 cores).
"""
import numpy as np
import pytest

from helpers import AGREE_MIN, DEN_MIN, TAU_TIE, TOL_DSUB, run_gpu, run_oracle
from paper_1807_07433_gb300 import synth

pytestmark = pytest.mark.gpu

WANT = ("lbl_l", "lbl_r", "gap_l", "gap_r", "den_l", "valid", "dfull")


@pytest.mark.parametrize("w", [synth.C2, synth.C3], ids=lambda w: w.name)
def test_full_frame_gate(w):
    from paper_1807_07433_gb300 import sr
    left, right, _ = synth.make_pair(w.scene)
    g = run_gpu(w, left, right, buffers=(("lbl_r", sr.SR_BUF_WTA_R),))
    o = run_oracle(w, left, right, WANT)
    H, W = left.shape

    diff = g["wta"].astype(np.int64) != o.lbl_l
    n_diff = int(diff.sum())
    n_hard = int((diff & (o.gap_l >= TAU_TIE)).sum())
    agree = 1.0 - n_diff / diff.size
    print(f"{w.name}: {n_diff} of {diff.size} labels differ ({100 * (1 - agree):.4f} %), "
          f"{n_hard} outside near-ties")
    assert n_hard == 0
    assert agree >= AGREE_MIN

    gfin = np.isfinite(g["dfull"])
    sharp = ~diff & (o.gap_l >= TAU_TIE) & (np.abs(o.den_l) >= DEN_MIN) & \
        np.isfinite(o.dfull) & gfin
    err = np.abs(g["dfull"][sharp] - o.dfull[sharp])
    print(f"{w.name}: subpixel checked at {int(sharp.sum())} pixels, max |dd| "
          f"{err.max():.2e} px, rms {np.sqrt(np.mean(err ** 2)):.2e} px; "
          f"{int((~diff & (np.abs(o.den_l) < DEN_MIN)).sum())} ill-conditioned parabolas skipped")
    assert sharp.mean() > 0.9
    assert err.max() <= TOL_DSUB

    # Eq. 11: validity is fixed by the labels at the pixel and at its match
    uu = np.arange(W)[None, :] - o.lbl_l
    inb = uu >= 0
    vv = np.broadcast_to(np.arange(H)[:, None], (H, W))
    match_same = np.ones((H, W), bool)
    match_same[inb] = g["lbl_r"][vv[inb], uu[inb]] == o.lbl_r[vv[inb], uu[inb]]
    firm = ~diff & match_same
    np.testing.assert_array_equal(gfin[firm], o.valid.astype(bool)[firm])
    assert firm.mean() > 0.99
