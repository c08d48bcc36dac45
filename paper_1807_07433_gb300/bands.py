"""Row-band partition of one frame over several GPUs, one band per rank.

Every step of the disparity path is local in the row direction up to a
window: the perspective transformation shifts each row on its own (Sec.
II-A), an NCC block spans 2*ncc_r + 1 rows (Eqs. 3-5), a bilateral window
2*agg_r + 1 rows of costs (Eqs. 8-10), and the L-R check and the
post-processing stay in the pixel's row (Eq. 11, Sec. II-C).  A band of
output rows [y0, y1) therefore needs only h = ncc_r + agg_r halo rows of both
images on either side, and the bands need no exchange: each rank holds its
rows r0..r1-1 and writes its own output rows (sr_match_rows).

The one quantity that crosses bands is the gradient of the aggregated cost
with respect to the road plane (sr_grad_plane): each band's share of L and of
dL/dalpha is summed over the ranks by one all-reduce of three FP64 values.

Host bookkeeping only: which rows each rank owns and reads, the plane of a
band that is handled as an image of its own, and the gradient reduction.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Band:
    y0: int          # first output row of the band
    y1: int          # one past its last output row
    r0: int          # first image row it reads (band + halo, clipped to the frame)
    r1: int          # one past the last image row it reads

    @property
    def rows(self) -> int:
        return self.y1 - self.y0

    @property
    def read_rows(self) -> int:
        return self.r1 - self.r0


def halo(ncc_r: int, agg_r: int) -> int:
    """Rows above and below a band that its NCC blocks and bilateral windows
    reach: ncc_r + agg_r."""
    return int(ncc_r) + int(agg_r)


def plan(H: int, n: int, ncc_r: int, agg_r: int, read_rows=None) -> list[Band]:
    """Split H rows into n bands of floor(H/n) or ceil(H/n) rows (the first
    H mod n bands take one more), each with its halo rows: by default the
    h = ncc_r + agg_r rows the windows reach; read_rows(y0, y1) -> (r0, r1)
    gives them instead where the matcher needs more (the GPU library's
    sr_band_rows, whose NCC kernel keeps window sums per segment of rows and
    so reads back to the start of a segment)."""
    if n < 1 or H < n:
        raise ValueError(f"cannot split {H} rows into {n} non-empty bands")
    h = halo(ncc_r, agg_r)
    base, extra = divmod(H, n)
    out, y = [], 0
    for k in range(n):
        rows = base + (1 if k < extra else 0)
        y0, y1 = y, y + rows
        r0, r1 = read_rows(y0, y1) if read_rows else (max(0, y0 - h), min(H, y1 + h))
        if not (0 <= r0 <= max(0, y0 - h) and r1 == min(H, y1 + h)):
            raise ValueError(f"rows [{r0}, {r1}) do not hold band [{y0}, {y1}) and its halo")
        out.append(Band(y0, y1, r0, r1))
        y = y1
    return out


def band_plane(alpha0: float, alpha1: float, r0: int) -> tuple[float, float]:
    """The plane (Eq. 2) of image rows r0.. seen as an image of their own,
    whose row v is row r0 + v of the frame: (alpha0 + alpha1 r0, alpha1).
    (sr_match_rows takes the frame's plane and its row offset instead, so
    that its results equal the frame's bit for bit.)"""
    return alpha0 + alpha1 * r0, alpha1


def frame_gradient(g_band, r0: int) -> np.ndarray:
    """dL/d(alpha0, alpha1) of the frame's plane from the gradient taken with
    respect to a band's own plane (band_plane): alpha0' = alpha0 + alpha1 r0,
    so dL/dalpha0 = dL/dalpha0' and dL/dalpha1 = dL/dalpha1' + r0 dL/dalpha0'."""
    g = np.asarray(g_band, dtype=np.float64)
    return np.array([g[0], g[1] + r0 * g[0]])


def allreduce_objective(L: float, g_frame, group=None) -> tuple[float, np.ndarray]:
    """Sum a band's share of L and dL/dalpha (frame coordinates) over the
    ranks of group: one all-reduce of three FP64 values."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(L), float(g_frame[0]), float(g_frame[1])], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized():
        if dist.get_backend(group) == "nccl":        # NCCL reduces device tensors
            t = t.to(torch.device("cuda", torch.cuda.current_device()))
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    v = t.cpu().numpy()
    return float(v[0]), v[1:].copy()
