"""Batched form: sr_match_batch over pairs of mixed sizes equals sr_match on
each pair (same tile kernels, so the results are bit-identical), across graph
replays, schedules chosen by the autotuner, and FP16 volumes; and each pair
of a mixed-size batch agrees with the FP64 oracle at the tolerances of the
single-pair parity tests."""
import numpy as np
import pytest

from paper_1807_07433_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [(97, 45), (160, 120), (203, 77), (64, 33), (160, 120), (31, 9)]
D, NCC_R, AGG_R, GD, GR = 32, 2, 3, 3.0, 10.0


def _pairs(seed0):
    out = []
    for k, (W, H) in enumerate(SIZES):
        sc = synth.Scene(W, H, 8.0 + k, 0.03 + 0.01 * k, 2, False, seed0 + k)
        left, right, _ = synth.make_pair(sc)
        out.append((left, right, sc.alpha0, sc.alpha1, 6.0 + (k % 3)))
    return out


def _single(pairs, vt):
    import torch
    from paper_1807_07433_gb300 import sr
    res = []
    for left, right, a0, a1, dl in pairs:
        H, W = left.shape
        with sr.Matcher(W, H, D, NCC_R, AGG_R, GD, GR, vol_dtype=vt,
                        stream=torch.cuda.current_stream()) as m:
            m.set_plane(a0, a1, dl)
            wta = torch.empty((H, W), dtype=torch.int16, device="cuda")
            disp = m.match(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(), wta=wta)
            torch.cuda.synchronize()
            res.append((disp.cpu().numpy(), wta.cpu().numpy()))
    return res


def _batch(ctx, pairs, order=None):
    import torch
    from paper_1807_07433_gb300 import sr
    order = list(range(len(pairs))) if order is None else order
    keep, descs, outs = [], [], {}
    for i in order:
        left, right, a0, a1, dl = pairs[i]
        H, W = left.shape
        tl, tr = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
        disp = torch.full((H, W), -3.0, device="cuda")
        wta = torch.full((H, W), -3, dtype=torch.int16, device="cuda")
        keep += [tl, tr]
        outs[i] = (disp, wta)
        descs.append(sr.make_pair_desc(tl, tr, disp, a0, a1, dl, wta))
    sr.sr_match_batch(ctx, descs)
    sr.sr_synchronize(ctx)
    return {i: (d.cpu().numpy(), w.cpu().numpy()) for i, (d, w) in outs.items()}


def _same(got, want):
    for i, (d, w) in want.items() if isinstance(want, dict) else enumerate(want):
        gd, gw = got[i]
        np.testing.assert_array_equal(gw, w)
        np.testing.assert_array_equal(np.isnan(gd), np.isnan(d))
        fin = np.isfinite(d)
        np.testing.assert_array_equal(gd[fin], d[fin])


def _check_pair_against_oracle(left, right, a0, a1, dl, disp, wta):
    """One pair of a batch against oracle.match (Eqs. 3, 8-12, Sec. II-C):
    labels differ only at near-ties, the full disparity is within TOL_DSUB
    where well conditioned, and validity (Eq. 11) is the oracle's wherever
    the labels agree at the pixel and the target view is not a near-tie at
    its match."""
    import oracle
    from helpers import AGREE_MIN, DEN_MIN, TAU_TIE, TOL_DSUB
    H, W = left.shape
    p = oracle.Params(W=W, H=H, D=D, ncc_r=NCC_R, agg_r=AGG_R, gamma_d=GD, gamma_r=GR,
                      lr_thresh=1.0, alpha0=a0, alpha1=a1, delta=dl)
    o = oracle.match(p, left, right, want=("lbl_l", "lbl_r", "gap_l", "gap_r", "den_l",
                                           "valid", "dfull"))
    diff = wta.astype(np.int64) != o.lbl_l
    assert not np.any(diff & (o.gap_l >= TAU_TIE)), (W, H)
    if W * H >= 5000:
        assert 1.0 - diff.mean() >= AGREE_MIN
    fin = np.isfinite(disp)
    sharp = ~diff & (o.gap_l >= TAU_TIE) & (np.abs(o.den_l) >= DEN_MIN) & \
        np.isfinite(o.dfull) & fin
    if sharp.any():
        assert np.abs(disp[sharp] - o.dfull[sharp]).max() <= TOL_DSUB
    uu = np.arange(W)[None, :] - o.lbl_l
    inb = uu >= 0
    vv = np.broadcast_to(np.arange(H)[:, None], (H, W))
    firm_match = np.ones((H, W), bool)
    firm_match[inb] = o.gap_r[vv[inb], uu[inb]] >= TAU_TIE
    firm = ~diff & firm_match
    np.testing.assert_array_equal(fin[firm], o.valid.astype(bool)[firm])


@pytest.mark.parametrize("variant", [0, 7])
def test_batch_matches_the_oracle(variant):
    """Every pair of a six-pair batch of mixed sizes (31x9 to 203x77) against
    the oracle, for a persistent schedule and the per-pair schedule."""
    from paper_1807_07433_gb300 import sr
    pairs = _pairs(700)
    with _ctx() as m:
        sr.sr_set_batch_schedule(m.ctx, variant)
        got = _batch(m.ctx, pairs)
    for i, (left, right, a0, a1, dl) in enumerate(pairs):
        _check_pair_against_oracle(left, right, a0, a1, dl, *got[i])


def _ctx(vt=0):
    import torch
    from paper_1807_07433_gb300 import sr
    return sr.Matcher(8, 8, D, NCC_R, AGG_R, GD, GR, vol_dtype=vt,
                      stream=torch.cuda.current_stream())


@pytest.mark.parametrize("vt", [0, 1])
def test_batch_equals_single_calls_and_replays(vt):
    from paper_1807_07433_gb300 import sr
    p1, p2 = _pairs(100), _pairs(200)
    with _ctx(vt) as m:
        _same(_batch(m.ctx, p1), _single(p1, vt))
        # graph replay with new images, planes and a new pair order
        _same(_batch(m.ctx, p2, order=[5, 3, 1, 0, 2, 4]), _single(p2, vt))
        info = sr.sr_batch_info(m.ctx)
        assert info["pairs"] == len(SIZES) and info["schedule"] == "persistent"


@pytest.mark.parametrize("variant", [1, 2, 4, 5, 6, 7])
def test_every_schedule_equals_single_calls(variant):
    from paper_1807_07433_gb300 import sr
    p1, p2 = _pairs(500), _pairs(600)
    with _ctx() as m:
        sr.sr_set_batch_schedule(m.ctx, variant)
        _same(_batch(m.ctx, p1), _single(p1, 0))
        _same(_batch(m.ctx, p2, order=[2, 0, 1, 5, 4, 3]), _single(p2, 0))
        info = sr.sr_batch_info(m.ctx)
        assert info["variant"] == variant
        assert info["schedule"] == ("per-pair-direct" if variant >= 6 else
                                    "per-pair-streams" if variant >= 4 else "persistent")
        with pytest.raises(sr.SrError):
            sr.sr_set_batch_schedule(m.ctx, 8)


def test_autotune_cache_round_trip(tmp_path):
    from paper_1807_07433_gb300 import sr
    cache = str(tmp_path / "tune.jsonl")
    p = _pairs(300)
    want = _single(p, 0)
    with _ctx() as m:
        sr.sr_set_autotune(m.ctx, True, cache)
        _same(_batch(m.ctx, p), want)
        info = sr.sr_batch_info(m.ctx)
        assert min(info["tune_ms"]) > 0.0          # every candidate was timed
        assert len(info["tune_ms"]) == 8
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and '"variant": %d' % info["variant"] in lines[0]
    with _ctx() as m:                               # a new context reuses the choice
        sr.sr_set_autotune(m.ctx, True, cache)
        _same(_batch(m.ctx, p), want)
        info2 = sr.sr_batch_info(m.ctx)
        assert info2["variant"] == info["variant"] and max(info2["tune_ms"]) == 0.0


def test_corrupted_tune_cache_falls_back_and_reports(tmp_path):
    from paper_1807_07433_gb300 import sr
    cache = tmp_path / "tune.jsonl"
    cache.write_text('{"key": "x", "variant": 99}\nnot json at all\n')
    p = _pairs(400)
    with _ctx() as m:
        sr.sr_set_autotune(m.ctx, True, str(cache))
        assert b"unreadable" in sr.load().sr_last_error(m.ctx)
        _same(_batch(m.ctx, p), _single(p, 0))


def test_batch_rejects_bad_pairs():
    import torch
    from paper_1807_07433_gb300 import sr
    t = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    d = torch.empty((8, 8), device="cuda")
    with _ctx() as m:
        bad = sr.make_pair_desc(t, t, d, 1.0, 0.0, 0.0)
        bad.pitch_bytes = 4
        with pytest.raises(sr.SrError) as e:
            sr.sr_match_batch(m.ctx, [bad])
        assert e.value.status == sr.SR_ERR_INVALID_ARG


@pytest.mark.parametrize("vt", [0, 1])
def test_batch_at_the_mixed_workload_sizes(vt):
    """One pair at each frame size of the 64-pair workload (672x376, 1280x720,
    1920x1080, 2208x1242), D = 64, NCC 7x7, bilateral 11x11, planes drawn as
    in that workload: the batch (tuned schedule) equals sr_match per pair bit
    for bit, FP32 and FP16 volumes."""
    import torch
    from paper_1807_07433_gb300 import sr
    rng = np.random.default_rng(1000)
    pairs = []
    for k, (W, H) in enumerate([(672, 376), (1280, 720), (1920, 1080), (2208, 1242)]):
        sc = synth.Scene(W, H, float(rng.uniform(10, 40)), float(rng.uniform(0.02, 0.1)), 20,
                         True, 1000 + k)
        left, right, _ = synth.make_pair(sc)
        pairs.append((left, right, sc.alpha0, sc.alpha1, 8.0))
    want = []
    for left, right, a0, a1, dl in pairs:
        H, W = left.shape
        with sr.Matcher(W, H, 64, 3, 5, 4.0, 12.0, vol_dtype=vt,
                        stream=torch.cuda.current_stream()) as m:
            m.set_plane(a0, a1, dl)
            wta = torch.empty((H, W), dtype=torch.int16, device="cuda")
            disp = m.match(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(), wta=wta)
            torch.cuda.synchronize()
            want.append((disp.cpu().numpy(), wta.cpu().numpy()))
    with sr.Matcher(8, 8, 64, 3, 5, 4.0, 12.0, vol_dtype=vt,
                    stream=torch.cuda.current_stream()) as m:
        sr.sr_set_autotune(m.ctx, True)
        _same(_batch(m.ctx, pairs), want)
        _same(_batch(m.ctx, pairs, order=[3, 1, 0, 2]), want)
        info = sr.sr_batch_info(m.ctx)
        if info["variant"] >= 6:
            # one slot per stream, each at most the largest pair's arrays
            e = 4 if vt == sr.SR_VOL_F32 else 2
            W, H = 2208, 1242
            slot = 2 * W * H * 4 + 4 * H * (W + 63) * 4 + H * (W + 63) * 64 * e + 2 * W * H * 2 + H * 8
            streams = min(info["streams"], len(pairs))
            assert info["scratch_bytes"] <= streams * (slot + 16 * 256), info


def test_scratch_is_bounded_by_streams_not_pairs():
    """Twelve small pairs under the 4-stream schedule of sr_match's kernels
    (7) take four slots of scratch; the persistent schedule (0) one per pair;
    the results are the same."""
    import torch
    from paper_1807_07433_gb300 import sr
    pairs = []
    for k in range(12):
        sc = synth.Scene(96 + 8 * (k % 3), 40, 12.0, 0.05, 1, False, 2000 + k)
        left, right, _ = synth.make_pair(sc)
        pairs.append((left, right, sc.alpha0, sc.alpha1, 8.0))
    with sr.Matcher(8, 8, 64, 2, 3, 3.0, 10.0, stream=torch.cuda.current_stream()) as m:
        sr.sr_set_batch_schedule(m.ctx, 0)
        out0 = _batch(m.ctx, pairs)
        s0 = sr.sr_batch_info(m.ctx)["scratch_bytes"]
        sr.sr_set_batch_schedule(m.ctx, 7)
        out7 = _batch(m.ctx, pairs)
        s7 = sr.sr_batch_info(m.ctx)["scratch_bytes"]
    _same(out7, out0)
    # four slots of the largest pair (widths 96..112) against twelve slots
    assert s7 <= 4 * (s0 / 12) * 1.2, (s7, s0)


def test_autotune_cache_path_from_environment(tmp_path, monkeypatch):
    """sr_set_autotune without a path takes SR_TUNE_CACHE from the environment."""
    from paper_1807_07433_gb300 import sr
    cache = tmp_path / "env_tune.jsonl"
    monkeypatch.setenv("SR_TUNE_CACHE", str(cache))
    p = _pairs(800)
    with _ctx() as m:
        sr.sr_set_autotune(m.ctx, True)
        _same(_batch(m.ctx, p), _single(p, 0))
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and '"variant"' in lines[0]
