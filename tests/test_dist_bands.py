"""The row-band partition of one frame over two ranks, on CPU (gloo,
127.0.0.1), with the FP64 oracle as each rank's matcher.

Each rank holds only its band's image rows and halo rows (bands.plan), runs
the oracle on them as an image of its own (the band's plane from
bands.band_plane), keeps its band's output rows, and the ranks gather them:
the result equals the oracle on the whole frame.  For the adjoint, each rank
takes the gradient of its band's share of L (the aggregated reference cost
at the plane hypothesis, rows outside the band left out), converts it to the
frame's plane (bands.frame_gradient) and the ranks sum it with one FP64
all-reduce (bands.allreduce_objective): the sum equals the whole frame's L
and dL/dalpha.  The band's plane differs from the frame's only by FP64
rounding of alpha0 + alpha1 r0, so outputs agree to 1e-9 and labels
exactly; the plane is kept away from warp kinks (helpers.kink_free_alpha)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene():
    sys.path.insert(0, ROOT)
    sys.path.insert(0, TESTS)
    from helpers import kink_free_alpha
    from paper_1807_07433_gb300 import synth
    w = synth.small(96, 46, D=16, ncc_r=2, agg_r=3, seed=77, alpha1=0.05)
    left, right, _ = synth.make_pair(w.scene)
    a0 = kink_free_alpha(w.scene.alpha0, w.scene.alpha1, w.delta, 46, 1e-9, 1e-9)
    return w, left, right, a0


def _params(w, H, a0, a1):
    import oracle
    return oracle.Params(W=w.scene.W, H=H, D=w.D, ncc_r=w.ncc_r, agg_r=w.agg_r,
                         gamma_d=w.gamma_d, gamma_r=w.gamma_r, lr_thresh=w.lr_thresh,
                         alpha0=a0, alpha1=a1, delta=w.delta)


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    w, left, right, a0 = _scene()
    import oracle
    from paper_1807_07433_gb300 import bands
    dist.init_process_group("gloo", init_method="env://")
    try:
        H, W = left.shape
        b = bands.plan(H, ws, w.ncc_r, w.agg_r)[rank]
        lr, rr = left[b.r0:b.r1].copy(), right[b.r0:b.r1].copy()   # all this rank holds
        pa0, pa1 = bands.band_plane(a0, w.scene.alpha1, b.r0)
        p = _params(w, b.read_rows, pa0, pa1)
        o = oracle.match(p, lr, rr, want=("lbl_l", "dfull"))
        k0, k1 = b.y0 - b.r0, b.y1 - b.r0
        mine = torch.from_numpy(np.stack([o.lbl_l[k0:k1].astype(np.float64),
                                          o.dfull[k0:k1]]))
        # gather the bands (each rank's rows padded to the largest band)
        rows = max(x.rows for x in bands.plan(H, ws, w.ncc_r, w.agg_r))
        pad = torch.full((2, rows, W), np.nan, dtype=torch.float64)
        pad[:, :b.rows] = mine
        got = [torch.empty_like(pad) for _ in range(ws)]
        dist.all_gather(got, pad)
        # adjoint: the band's share of L at the plane hypothesis
        dstar = np.full((b.read_rows, W), -1, np.int32)
        dstar[k0:k1] = int(round(w.delta))
        L, g, _, _ = oracle.grad(p, lr.astype(np.float64), rr.astype(np.float64), dstar)
        Ls, gs = bands.allreduce_objective(L, bands.frame_gradient(g, b.r0))
        q.put((rank, [x.numpy() for x in got] if rank == 0 else None, Ls, gs))
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_a_frame_into_bands():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(ws)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0

    import oracle
    from paper_1807_07433_gb300 import bands
    w, left, right, a0 = _scene()
    H, W = left.shape
    full = oracle.match(_params(w, H, a0, w.scene.alpha1), left, right, want=("lbl_l", "dfull"))
    plan = bands.plan(H, ws, w.ncc_r, w.agg_r)
    assert plan[0].r0 == 0 and plan[-1].r1 == H and plan[0].y1 == plan[1].y0
    lbl = np.concatenate([res[0][1][k][0, :b.rows] for k, b in enumerate(plan)])
    dfull = np.concatenate([res[0][1][k][1, :b.rows] for k, b in enumerate(plan)])
    np.testing.assert_array_equal(lbl, full.lbl_l.astype(np.float64))
    np.testing.assert_array_equal(np.isnan(dfull), np.isnan(full.dfull))
    fin = np.isfinite(full.dfull)
    np.testing.assert_allclose(dfull[fin], full.dfull[fin], rtol=0, atol=1e-9)

    dstar = np.full((H, W), int(round(w.delta)), np.int32)
    L, g, _, _ = oracle.grad(_params(w, H, a0, w.scene.alpha1), left.astype(np.float64),
                             right.astype(np.float64), dstar)
    for _, _, Ls, gs in res:                   # every rank holds the same sums
        assert abs(Ls - L) <= 1e-9 * abs(L)
        np.testing.assert_allclose(gs, g, rtol=1e-8, atol=1e-9 * np.abs(g).max())


def test_plan_covers_the_frame_with_halos():
    sys.path.insert(0, ROOT)
    from paper_1807_07433_gb300 import bands
    for H, n, r, R in ((720, 4, 3, 5), (7, 7, 1, 1), (121, 3, 5, 7), (5, 2, 3, 4)):
        p = bands.plan(H, n, r, R)
        assert [b.y0 for b in p][0] == 0 and p[-1].y1 == H
        assert all(a.y1 == b.y0 for a, b in zip(p, p[1:]))
        assert max(b.rows for b in p) - min(b.rows for b in p) <= 1
        for b in p:
            assert b.r0 == max(0, b.y0 - (r + R)) and b.r1 == min(H, b.y1 + r + R)
    # rows read back to a segment start (the GPU library's rule), and a
    # read range that misses the halo is refused
    seg = 32
    rows = lambda y0, y1: (max(0, max(0, y0 - 5) // seg * seg - 3), min(720, y1 + 8))  # noqa: E731
    for b in bands.plan(720, 4, 3, 5, read_rows=rows):
        assert b.r0 <= max(0, b.y0 - 8) and b.r0 % seg in (0, seg - 3) and b.r1 == min(720, b.y1 + 8)
    with pytest.raises(ValueError):
        bands.plan(720, 4, 3, 5, read_rows=lambda y0, y1: (y0, y1))
    g = bands.frame_gradient([2.0, 3.0], 10)
    np.testing.assert_array_equal(g, [2.0, 23.0])
    assert bands.band_plane(30.0, 0.08, 100) == (30.0 + 8.0, 0.08)
