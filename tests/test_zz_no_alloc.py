"""sr_match_noalloc: the match for callers that cannot allocate device memory.

Such callers (a host that fixes the device-memory budget at start-up, a
plug-in whose host owns the allocator, a real-time loop that must not wait on
the allocator) get the same disparities as sr_match without creating a
context: the intermediates live in a fixed 32 MiB device array inside the
library.  This module runs last so that a failure here never hides one
elsewhere; it must pass on its own in a fresh process too.
"""
import numpy as np
import pytest

from helpers import TOL_DSUB
from paper_1807_07433_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [synth.C1, synth.small(203, 77, D=32, ncc_r=3, agg_r=5, seed=11),
         synth.small(150, 90, D=64, ncc_r=3, agg_r=5, seed=21, alpha1=0.08)]


def _reference(w, dl, dr, torch, sr):
    H, W = dl.shape
    with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                    stream=torch.cuda.current_stream()) as m:
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        wta = torch.empty((H, W), dtype=torch.int16, device="cuda")
        disp = m.match(dl, dr, wta=wta)
        torch.cuda.synchronize()
        return disp.cpu().numpy(), wta.cpu().numpy()


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_noalloc_matches_sr_match_on_two_calls_in_a_row(w):
    import torch
    from paper_1807_07433_gb300 import sr
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    dl = torch.from_numpy(left).cuda()
    dr = torch.from_numpy(right).cuda()
    ref_disp, ref_wta = _reference(w, dl, dr, torch, sr)
    params = sr.make_params(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh)
    for _ in range(2):
        disp = torch.full((H, W), -7.0, dtype=torch.float32, device="cuda")
        wta = torch.full((H, W), -7, dtype=torch.int16, device="cuda")
        sr.sr_match_noalloc(params, w.scene.alpha0, w.scene.alpha1, w.delta, dl, dr, W, disp,
                            wta, torch.cuda.current_stream())
        torch.cuda.synchronize()
        d, l = disp.cpu().numpy(), wta.cpu().numpy()
        np.testing.assert_array_equal(l, ref_wta)
        np.testing.assert_array_equal(np.isnan(d), np.isnan(ref_disp))
        fin = np.isfinite(ref_disp)
        np.testing.assert_allclose(d[fin], ref_disp[fin], rtol=0, atol=TOL_DSUB)


def test_noalloc_rejects_frames_beyond_its_scratch():
    import torch
    from paper_1807_07433_gb300 import sr
    params = sr.make_params(1280, 720, 64, 3, 5, 4.0, 12.0)
    buf = torch.zeros((720, 1280), dtype=torch.uint8, device="cuda")
    out = torch.empty((720, 1280), dtype=torch.float32, device="cuda")
    with pytest.raises(sr.SrError) as e:
        sr.sr_match_noalloc(params, 30.0, 0.08, 8.0, buf, buf, 1280, out)
    assert e.value.status == sr.SR_ERR_UNSUPPORTED
