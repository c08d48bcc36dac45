"""Seeded synthetic road scenes: the input generator shared by tests and bench.

The paper evaluates on ZED road footage and 3-D-printed sample models
(Sec. III), neither of which is available.  This module renders stand-ins
with the structure of those scenes: a textured road plane whose disparity
follows the linear model of Eq. 2, d(u,v) = alpha0 + alpha1*v, dented by
Gaussian potholes and thin crack-like grooves, seen by a rectified stereo pair
with sensor noise.  It holds scene synthesis only -- none of the matching
method's arithmetic -- so both the CUDA path's tests and the oracle's tests
can draw their inputs from it.

Recipe (all randomness from numpy PCG64 seeded per scene):
  * texture T(x,y): 4 octaves of value noise, lattice spacings 32/16/8/4 px,
    amplitudes 1, 1/2, 1/4, 1/8, lattice values U[-1,1], bilinear between
    lattice points (defined at any real x), rescaled to mean 128, std 40
    over the left image;
  * disparity d(u,v) = alpha0 + alpha1*v - min(2, potholes + grooves); a
    pothole is A*exp(-r^2/(2 s^2)) within 4 s of its centre, A ~ U[0.5,2],
    s ~ U[5,12] px; a groove is
    a random 3-segment polyline with a triangular profile 1-3 px wide and
    0.5-2 px deep;
  * left(u,v) = T(u,v); right(u_r,v) = T(u_l,v) with u_l = u_r + d(u_l,v)
    solved by 3 fixed-point steps; N(0, 2^2) noise on each image, rounded
    and clipped to uint8.
"""
from __future__ import annotations

from dataclasses import dataclass, asdict

import numpy as np

_OCTAVES = ((32.0, 1.0), (16.0, 0.5), (8.0, 0.25), (4.0, 0.125))


@dataclass(frozen=True)
class Scene:
    """Scene description; alpha0/alpha1 are the true Eq. 2 road-plane terms."""
    W: int
    H: int
    alpha0: float
    alpha1: float
    n_potholes: int
    grooves: bool
    seed: int
    noise_sigma: float = 2.0


@dataclass(frozen=True)
class Workload:
    """A matching workload: scene plus method parameters."""
    name: str
    scene: Scene
    D: int             # residual disparities searched, 0..D-1
    ncc_r: int         # NCC block radius (window 2r+1)
    agg_r: int         # bilateral radius (window 2r+1)
    gamma_d: float     # sigma_s of the workload, read as gamma_d of Eq. 9
    gamma_r: float     # sigma_r of the workload, read as gamma_r of Eq. 10
    delta: float       # offset of Sec. II-A keeping residual disparities >= 0
    lr_thresh: float = 1.0
    f_px: float = 700.0
    baseline_mm: float = 120.0

    def describe(self) -> dict:
        d = asdict(self)
        d["scene"] = asdict(self.scene)
        return d


def _lattice_noise(rng: np.random.Generator, x_max: float, y_max: float):
    """Lattice tables for each octave covering [0, x_max] x [0, y_max]."""
    tables = []
    for spacing, amp in _OCTAVES:
        nx = int(np.ceil(x_max / spacing)) + 3
        ny = int(np.ceil(y_max / spacing)) + 3
        tables.append((spacing, amp, rng.uniform(-1.0, 1.0, size=(ny, nx))))
    return tables


def _texture(tables, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Value-noise texture at real coordinates (x, y) >= 0 (float64)."""
    out = np.zeros(np.broadcast(x, y).shape, np.float64)
    for spacing, amp, tab in tables:
        gx = x / spacing
        gy = y / spacing
        ix = np.floor(gx).astype(np.int64)
        iy = np.floor(gy).astype(np.int64)
        fx = gx - ix
        fy = gy - iy
        v00 = tab[iy, ix]
        v01 = tab[iy, ix + 1]
        v10 = tab[iy + 1, ix]
        v11 = tab[iy + 1, ix + 1]
        top = v00 * (1.0 - fx) + v01 * fx
        bot = v10 * (1.0 - fx) + v11 * fx
        out += amp * (top * (1.0 - fy) + bot * fy)
    return out


def _depressions(rng: np.random.Generator, sc: Scene):
    """Pothole and groove parameters, drawn once per scene."""
    pots = []
    for _ in range(sc.n_potholes):
        pots.append((rng.uniform(0, sc.W), rng.uniform(0, sc.H), rng.uniform(0.5, 2.0),
                     rng.uniform(5.0, 12.0)))
    grooves = []
    if sc.grooves:
        n_g = max(1, sc.n_potholes // 4)
        for _ in range(n_g):
            pts = [(rng.uniform(0, sc.W), rng.uniform(0, sc.H))]
            ang = rng.uniform(0, 2 * np.pi)
            for _ in range(3):
                ang += rng.uniform(-0.6, 0.6)
                ln = rng.uniform(0.1, 0.3) * min(sc.W, sc.H)
                pts.append((pts[-1][0] + ln * np.cos(ang), pts[-1][1] + ln * np.sin(ang)))
            grooves.append((pts, rng.uniform(0.5, 1.5), rng.uniform(0.5, 2.0)))
    return pots, grooves


def _depth(u: np.ndarray, v: np.ndarray, pots, grooves) -> np.ndarray:
    """Total depression at points (u[r, c], row r); v[r, :] == r.  Each feature
    is evaluated on the rows it reaches (a pothole within 4 sigma, a groove
    within its segment's rows plus its half width)."""
    H = u.shape[0]
    dep = np.zeros(u.shape, np.float64)
    for (uk, vk, a, s) in pots:
        r0, r1 = max(0, int(vk - 4 * s)), min(H, int(vk + 4 * s) + 2)
        if r0 >= r1:
            continue
        uu, vv = u[r0:r1], v[r0:r1]
        dep[r0:r1] += a * np.exp(-((uu - uk) ** 2 + (vv - vk) ** 2) / (2.0 * s * s))
    for pts, half_w, depth in grooves:
        dist = np.full(dep.shape, np.inf)
        rows = np.zeros(H, bool)
        for (x0, y0), (x1, y1) in zip(pts[:-1], pts[1:]):
            r0 = max(0, int(min(y0, y1) - half_w) - 1)
            r1 = min(H, int(max(y0, y1) + half_w) + 2)
            if r0 >= r1:
                continue
            rows[r0:r1] = True
            uu, vv = u[r0:r1], v[r0:r1]
            ex, ey = x1 - x0, y1 - y0
            t = np.clip(((uu - x0) * ex + (vv - y0) * ey) / (ex * ex + ey * ey), 0.0, 1.0)
            dist[r0:r1] = np.minimum(dist[r0:r1],
                                     np.hypot(uu - (x0 + t * ex), vv - (y0 + t * ey)))
        if rows.any():
            dep[rows] += depth * np.clip(1.0 - dist[rows] / half_w, 0.0, None)
    return np.minimum(dep, 2.0)


def features(sc: Scene):
    """The scene's potholes [(u, v, depth_px, sigma_px)] and grooves, drawn in
    the order make_pair draws them (same generator state)."""
    rng = np.random.Generator(np.random.PCG64(sc.seed))
    d_hi = sc.alpha0 + sc.alpha1 * sc.H + 4.0
    _lattice_noise(rng, sc.W + d_hi + 8.0, sc.H + 2.0)
    return _depressions(rng, sc)


def make_pair(sc: Scene):
    """Render (left uint8 [H,W], right uint8 [H,W], true disparity float64 [H,W])."""
    rng = np.random.Generator(np.random.PCG64(sc.seed))
    d_hi = sc.alpha0 + sc.alpha1 * sc.H + 4.0
    tables = _lattice_noise(rng, sc.W + d_hi + 8.0, sc.H + 2.0)
    pots, grooves = _depressions(rng, sc)

    v, u = np.mgrid[0:sc.H, 0:sc.W].astype(np.float64)
    plane = sc.alpha0 + sc.alpha1 * v

    def disp(ul):
        return plane - _depth(ul, v, pots, grooves)

    d_true = disp(u)
    tex_l = _texture(tables, u, v)
    m, s = tex_l.mean(), tex_l.std()
    if not s > 0.0:          # a single pixel has no spread
        s = 1.0
    scale = lambda t: 128.0 + 40.0 * (t - m) / s  # noqa: E731

    ul = u + plane
    for _ in range(3):
        ul = u + disp(ul)
    tex_r = _texture(tables, ul, v)

    left = scale(tex_l) + rng.normal(0.0, sc.noise_sigma, size=tex_l.shape)
    right = scale(tex_r) + rng.normal(0.0, sc.noise_sigma, size=tex_r.shape)
    left = np.clip(np.rint(left), 0, 255).astype(np.uint8)
    right = np.clip(np.rint(right), 0, 255).astype(np.uint8)
    return left, right, d_true


# Workloads.  Parameters not given for a workload are taken from the
# 1280x720 one; delta is 4 for 16 disparities and 8 for 64.
C1 = Workload("plain-fp32 160x120 D16 ncc5 bil9",
              Scene(160, 120, 8.0, 0.05, 3, False, 1), D=16, ncc_r=2, agg_r=4,
              gamma_d=3.0, gamma_r=10.0, delta=4.0)
C2 = Workload("plain-fp32 1280x720 D64 ncc7 bil11",
              Scene(1280, 720, 30.0, 0.08, 20, True, 2), D=64, ncc_r=3, agg_r=5,
              gamma_d=4.0, gamma_r=12.0, delta=8.0)
C3 = Workload("precision 1920x1080 D64 ncc7 bil11",
              Scene(1920, 1080, 30.0, 0.08, 20, True, 3), D=64, ncc_r=3, agg_r=5,
              gamma_d=4.0, gamma_r=12.0, delta=8.0)

BATCH_SIZES = ((672, 376), (1280, 720), (1920, 1080), (2208, 1242))


def batch_workloads(n_per_size: int = 16):
    """Mixed-size batch: n_per_size pairs at each of four resolutions; pair k
    uses seed 1000+k and draws alpha0 ~ U[10,40], alpha1 ~ U[0.02,0.1]."""
    out = []
    k = 0
    for (W, H) in BATCH_SIZES:
        for _ in range(n_per_size):
            rng = np.random.Generator(np.random.PCG64(1000 + k))
            a0 = float(rng.uniform(10.0, 40.0))
            a1 = float(rng.uniform(0.02, 0.1))
            out.append(Workload(f"batch[{k}] {W}x{H}", Scene(W, H, a0, a1, 20, True, 1000 + k),
                                D=64, ncc_r=3, agg_r=5, gamma_d=4.0, gamma_r=12.0, delta=8.0))
            k += 1
    return out


def small(W: int, H: int, D: int = 16, ncc_r: int = 2, agg_r: int = 3, seed: int = 7,
          alpha0: float = 8.0, alpha1: float = 0.05, n_potholes: int = 2,
          gamma_d: float = 3.0, gamma_r: float = 10.0, delta: float | None = None) -> Workload:
    """A small workload for parity tests at arbitrary (ragged) sizes."""
    if delta is None:
        delta = 4.0 if D <= 16 else 8.0
    return Workload(f"small {W}x{H} D{D}", Scene(W, H, alpha0, alpha1, n_potholes, False, seed),
                    D=D, ncc_r=ncc_r, agg_r=agg_r, gamma_d=gamma_d, gamma_r=gamma_r, delta=delta)
