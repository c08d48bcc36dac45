"""Child process of tests/test_gpu_bounds.py: runs the match path with the
bounds-checked library (libsr_check.so) and saves its outputs and the bounds
reports to an .npz file named on the command line.

Cases: the stage-parity scenes (ragged, tiny and degenerate sizes), the
1280x720x64 benchmark frame at FP32 and FP16, the restricted search, the
row-band form and reconstruction; then the report self-test.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from paper_1807_07433_gb300 import bands, sr, synth  # noqa: E402

CASES = [
    ("c1", synth.C1, 0),
    ("r203", synth.small(203, 77, D=32, ncc_r=3, agg_r=5, seed=11), 0),
    ("r97", synth.small(97, 45, D=64, ncc_r=1, agg_r=7, seed=12, gamma_d=5.0, gamma_r=15.0), 0),
    ("r33", synth.small(33, 5, D=16, ncc_r=2, agg_r=3, seed=14), 0),
    ("r1", synth.small(1, 1, D=16, ncc_r=1, agg_r=1, seed=15), 0),
    ("r5", synth.small(5, 2, D=16, ncc_r=3, agg_r=4, seed=16), 0),
    ("r6", synth.small(6, 300, D=64, ncc_r=2, agg_r=4, seed=52, alpha1=0.01), 0),
    ("c2", synth.C2, 0),
    ("c2h", synth.C2, 1),
]


def run_case(w, vol_dtype):
    import torch
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    dl, dr = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    out = {}
    with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                    vol_dtype=vol_dtype, stream=torch.cuda.current_stream()) as m:
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        m.set_camera(w.f_px, w.baseline_mm)
        wta = torch.empty((H, W), dtype=torch.int16, device="cuda")
        disp = m.match(dl, dr, wta=wta)
        out["disp"] = disp.cpu().numpy()
        out["wta"] = wta.cpu().numpy()
        out["xyz"] = m.reconstruct(disp).cpu().numpy()
        if w.D == 64 and H >= 64:
            out["restricted"] = m.match_restricted(dl, dr, 4).cpu().numpy()
            rows = []
            for b in bands.plan(H, 3, w.ncc_r, w.agg_r, read_rows=m.band_rows):
                rows.append(m.match_rows(dl[b.r0:b.r1].contiguous(), dr[b.r0:b.r1].contiguous(),
                                         b.y0, b.y1).cpu().numpy())
            out["rows"] = np.concatenate(rows)
        torch.cuda.synchronize()
    return out


BATCH_SIZES = [(96, 40), (203, 77), (150, 61)]
BATCH_VARIANTS = (0, 4, 7)   # persistent, descriptor-driven per pair, sr_match's kernels


def run_batch(variant):
    """A mixed-size batch (D = 64, FP32) under one schedule, then one plain
    match (launches inside the batch's graph are checked by the next plain
    launch of their kernel files); returns the pairs' outputs."""
    import torch
    keep, descs, outs = [], [], []
    for k, (W, H) in enumerate(BATCH_SIZES):
        sc = synth.Scene(W, H, 12.0 + k, 0.05, 1, False, 3000 + k)
        left, right, _ = synth.make_pair(sc)
        tl, tr = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
        disp = torch.full((H, W), -3.0, device="cuda")
        wta = torch.full((H, W), -3, dtype=torch.int16, device="cuda")
        keep += [tl, tr]
        outs.append((disp, wta))
        descs.append(sr.make_pair_desc(tl, tr, disp, sc.alpha0, sc.alpha1, 8.0, wta))
    with sr.Matcher(8, 8, 64, 3, 5, 4.0, 12.0, stream=torch.cuda.current_stream()) as m:
        sr.sr_set_batch_schedule(m.ctx, variant)
        sr.sr_match_batch(m.ctx, descs)
        sr.sr_match_batch(m.ctx, descs)   # a replay of the graph
        sr.sr_synchronize(m.ctx)
    w = synth.small(64, 16, D=64, ncc_r=3, agg_r=5, seed=3100)
    left, right, _ = synth.make_pair(w.scene)
    with sr.Matcher(64, 16, 64, 3, 5, 4.0, 12.0, stream=torch.cuda.current_stream()) as m:
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        m.match(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda())
        torch.cuda.synchronize()
    res = {}
    for k, (d, wt) in enumerate(outs):
        res[f"disp{k}"] = d.cpu().numpy()
        res[f"wta{k}"] = wt.cpu().numpy()
    return res


def main(path):
    import torch
    sr.load(sr.CHECK_LIB_PATH)
    torch.cuda.set_device(0)
    res = {}
    for name, w, vt in CASES:
        for k, v in run_case(w, vt).items():
            res[f"{name}.{k}"] = v
        st, site, index, unit, count = sr.sr_bounds_report()
        res[f"{name}.report"] = np.array([st, site, index, count], dtype=np.int64)
    for v in BATCH_VARIANTS:
        for k, a in run_batch(v).items():
            res[f"batch{v}.{k}"] = a
        st, site, index, unit, count = sr.sr_bounds_report()
        res[f"batch{v}.report"] = np.array([st, site, index, count], dtype=np.int64)
    # self-test: one recorded offence (site 399, index -1), no memory access
    w = synth.C1
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                    stream=torch.cuda.current_stream()) as m:
        m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
        m.set_camera(w.f_px, w.baseline_mm)
        disp = m.match(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda())
        sr.sr_set_debug(m.ctx, sr.SR_DEBUG_BOUNDS_SELFTEST)
        status = sr.SR_OK
        try:
            m.reconstruct(disp)
        except sr.SrError as e:
            status = e.status
        st, site, index, unit, count = sr.sr_bounds_report()
        res["selftest.call_status"] = np.array(status)
        res["selftest.report"] = np.array([st, site, index, count], dtype=np.int64)
        res["selftest.unit"] = np.array(unit)
        sr.sr_set_debug(m.ctx, 0)
        m.reconstruct(disp)   # and the context goes on
        torch.cuda.synchronize()
        st, site, index, _, count = sr.sr_bounds_report()
        res["after.report"] = np.array([st, site, index, count], dtype=np.int64)
    np.savez(path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
