"""Row bands of one frame as virtual shards on one GPU: sr_match_rows on
2, 3 and 4 bands (each from its own rows and halo rows only, as
sr_band_rows gives them) gives the
disparity and label maps of one sr_match on the whole frame, bit for bit.
The bands are planned by paper_1807_07433_gb300.bands, the partition a
multi-GPU run uses (one band per rank)."""
import math

import numpy as np
import pytest

from paper_1807_07433_gb300 import bands, synth

pytestmark = pytest.mark.gpu

SCENES = [synth.C1, synth.small(203, 77, D=32, ncc_r=3, agg_r=5, seed=11),
          synth.small(97, 45, D=64, ncc_r=1, agg_r=7, seed=12), synth.C2]


def _full(m, dl, dr, torch):
    H, W = dl.shape
    wta = torch.empty((H, W), dtype=torch.int16, device="cuda")
    disp = m.match(dl, dr, wta=wta)
    torch.cuda.synchronize()
    return disp.cpu().numpy(), wta.cpu().numpy()


@pytest.mark.parametrize("w", SCENES, ids=lambda w: w.name)
def test_bands_equal_the_whole_frame(w):
    import torch
    from paper_1807_07433_gb300 import sr
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    dl, dr = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                    stream=torch.cuda.current_stream()) as m:
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        want_d, want_l = _full(m, dl, dr, torch)
        for n in (2, 3, 4):
            got_d = np.full((H, W), -5.0, np.float32)
            got_l = np.full((H, W), -5, np.int16)
            for b in bands.plan(H, n, w.ncc_r, w.agg_r, read_rows=m.band_rows):
                # the band sees only its own rows and halo rows
                lr = dl[b.r0:b.r1].clone()
                rr = dr[b.r0:b.r1].clone()
                wta = torch.empty((b.rows, W), dtype=torch.int16, device="cuda")
                d = m.match_rows(lr, rr, b.y0, b.y1, wta_rows=wta)
                torch.cuda.synchronize()
                got_d[b.y0:b.y1] = d.cpu().numpy()
                got_l[b.y0:b.y1] = wta.cpu().numpy()
            np.testing.assert_array_equal(got_l, want_l)
            np.testing.assert_array_equal(got_d.view(np.uint32), want_d.view(np.uint32))
        # the whole frame as one band, and single rows at both ends
        d = m.match_rows(dl, dr, 0, H)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32), want_d.view(np.uint32))
        for y in (0, H - 1):
            b = [x for x in bands.plan(H, H, w.ncc_r, w.agg_r, read_rows=m.band_rows)
                 if x.y0 == y][0]
            d = m.match_rows(dl[b.r0:b.r1].clone(), dr[b.r0:b.r1].clone(), b.y0, b.y1)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32),
                                          want_d[y:y + 1].view(np.uint32))


def test_band_arguments_are_checked():
    import torch
    from paper_1807_07433_gb300 import sr
    buf = torch.zeros((32, 64), dtype=torch.uint8, device="cuda")
    out = torch.empty((32, 64), device="cuda")
    with sr.Matcher(64, 32, 16, 2, 2, 3.0, 10.0) as m:
        for y0, y1 in ((-1, 4), (4, 4), (10, 33)):
            with pytest.raises(sr.SrError) as e:
                sr.sr_match_rows(m.ctx, buf, buf, 64, y0, y1, out)
            assert e.value.status == sr.SR_ERR_INVALID_ARG


def test_band_rows_cover_the_halo_and_start_a_segment():
    """sr_band_rows: r1 = min(H, y1 + h) and r0 <= y0 - h (or 0); every band's
    r0 + ncc_r is a multiple of one segment length (or r0 = 0)."""
    from paper_1807_07433_gb300 import sr
    W, H, r, R = 1280, 720, 3, 5
    with sr.Matcher(W, H, 64, r, R, 4.0, 12.0) as m:
        starts = set()
        for y0 in range(0, H, 37):
            y1 = min(H, y0 + 50)
            r0, r1 = m.band_rows(y0, y1)
            assert r1 == min(H, y1 + r + R)
            assert 0 <= r0 <= max(0, y0 - r - R)
            if r0 > 0:
                starts.add(r0 + r)
        g = 0
        for s0 in starts:
            g = math.gcd(g, s0)
        assert g >= 8, sorted(starts)   # segments of at least 8 rows
        with pytest.raises(sr.SrError):
            m.band_rows(5, 5)
