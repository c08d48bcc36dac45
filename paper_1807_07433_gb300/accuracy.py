"""Synthetic analogue of the sample-model experiment of Sec. III.

The paper measures 3-D-printed models of known depth with its pipeline and
reports an accuracy of about 3 mm.  Here the synthetic road scenes carry
Gaussian potholes of known depth: for every pothole clear of the other
depressions and of the frame border, a road plane is fitted (least squares)
to the reconstructed 3-D points of a ring around it (4 to 6 sigma), and the
distance to that plane of the reconstructed points near its bottom (within
sigma / 2) is the measured depth.  The same construction on the generator's
true disparity gives the true depth; the error is measured minus true depth,
in the length unit of the baseline (mm).  Host evaluation of the 3-D points
of Sec. II-D; it holds none of the matching arithmetic.
"""
from __future__ import annotations

import numpy as np


def _groove_mask(grooves, H: int, W: int, margin: float = 3.0) -> np.ndarray:
    vv, uu = np.mgrid[0:H, 0:W].astype(np.float64)
    mask = np.zeros((H, W), bool)
    for pts, half_w, _ in grooves:
        for (x0, y0), (x1, y1) in zip(pts[:-1], pts[1:]):
            ex, ey = x1 - x0, y1 - y0
            t = np.clip(((uu - x0) * ex + (vv - y0) * ey) / (ex * ex + ey * ey), 0.0, 1.0)
            mask |= np.hypot(uu - (x0 + t * ex), vv - (y0 + t * ey)) < half_w + margin
    return mask


def _plane_dist(P: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """Distances of points Q (N x 3) to the least-squares plane of P (M x 3)."""
    c = P.mean(0)
    n = np.linalg.svd(P - c, full_matrices=False)[2][-1]
    return np.abs((Q - c) @ n)


def true_points(d_true: np.ndarray, f: float, B: float, u0: float, v0: float) -> np.ndarray:
    """The 3-D points [3, H, W] of the true disparity (Sec. II-D projection)."""
    H, W = d_true.shape
    vv, uu = np.mgrid[0:H, 0:W].astype(np.float64)
    Z = f * B / d_true
    return np.stack([(uu - u0) * Z / f, (vv - v0) * Z / f, Z])


def pothole_depths(xyz: np.ndarray, d_true: np.ndarray, scene, pots, grooves, f: float,
                   B: float, u0: float, v0: float, usable: np.ndarray | None = None) -> list[dict]:
    """Measured and true depth of every isolated pothole.

    xyz: reconstructed points [3, H, W] (NaN where rejected); usable: optional
    [H, W] mask of the points the evaluation may use (default: finite)."""
    H, W = d_true.shape
    xyz = np.asarray(xyz, dtype=np.float64)
    xyz_t = true_points(d_true, f, B, u0, v0)
    vv, uu = np.mgrid[0:H, 0:W].astype(np.float64)
    groove = _groove_mask(grooves, H, W)
    ok_pts = np.isfinite(xyz[2]) if usable is None else (usable & np.isfinite(xyz[2]))
    rows = []
    for k, (uk, vk, a, s) in enumerate(pots):
        if not (6 * s <= uk < W - 6 * s and 6 * s <= vk < H - 6 * s):
            continue
        if any(j != k and np.hypot(uk - uj, vk - vj) < 6 * s + 4 * sj
               for j, (uj, vj, _, sj) in enumerate(pots)):
            continue
        r = np.hypot(uu - uk, vv - vk)
        ring = (r >= 4 * s) & (r <= 6 * s) & ~groove
        core = (r <= 0.5 * s) & ~groove
        if groove[(r <= 6 * s)].any() or \
                (d_true[core] <= scene.alpha0 + scene.alpha1 * vv[core] - 2.0).any():
            continue
        ok_ring, ok_core = ring & ok_pts, core & ok_pts
        if ok_ring.sum() < 50 or ok_core.sum() < 5:
            continue
        meas = _plane_dist(xyz[:, ok_ring].T, xyz[:, ok_core].T)
        true = _plane_dist(xyz_t[:, ok_ring].T, xyz_t[:, ok_core].T)
        err = meas - true
        rows.append({"pothole": k, "u": round(float(uk), 1), "v": round(float(vk), 1),
                     "depth_px": round(float(a), 3), "sigma_px": round(float(s), 2),
                     "true_depth_mm": float(true.mean()), "measured_depth_mm": float(meas.mean()),
                     "error_mm_mean": float(err.mean()),
                     "error_mm_rms": float(np.sqrt((err ** 2).mean())),
                     "points": int(ok_core.sum())})
    return rows
