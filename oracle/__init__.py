"""FP64 CPU oracle for the road-surface stereo hot path (arXiv 1807.07433).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
and the benchmark's CPU-baseline / reference arm may import this package.
The CUDA path never imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, double precision, direct
definitions of Eqs. 2-12 and Secs. II-A..II-D); this module only compiles it
with gcc and marshals numpy arrays through ctypes.

Every function here is pinned by ``tests/test_oracle_pins.py`` against facts
the paper and mathematics fix (library routines, closed forms, invariants,
brute force).  Parity status per function is listed in that test module's
docstring; nothing here is "parity unpinned" except the synthetic scenes'
ground truth, which is not an oracle function.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, out: str | None = None, mutant: int = 0) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no FMA contraction);
    with mutant k > 0, into out with planted mistake k (pin tests only)."""
    if mutant:
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", f"-DORC_MUTANT={int(mutant)}", _SRC, "-o", out, "-lm"]
        subprocess.run(cmd, check=True)
        return out
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("D", ctypes.c_int),
                ("ncc_r", ctypes.c_int), ("agg_r", ctypes.c_int),
                ("gamma_d", ctypes.c_double), ("gamma_r", ctypes.c_double),
                ("lr_thresh", ctypes.c_double),
                ("alpha0", ctypes.c_double), ("alpha1", ctypes.c_double),
                ("delta", ctypes.c_double),
                ("f_px", ctypes.c_double), ("baseline", ctypes.c_double),
                ("u0", ctypes.c_double), ("v0", ctypes.c_double)]


_P = ctypes.c_void_p


class _Outputs(ctypes.Structure):
    _fields_ = [(n, _P) for n in (
        "warped", "mu_l", "sig_l", "mu_r", "sig_r", "cost_l", "cost_r",
        "agg_l", "agg_r", "lbl_l", "lbl_r", "gap_l", "gap_r", "den_l",
        "dsub", "valid", "dfull", "xyz")]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # ORC_LIB: a library built from oracle.c with a planted mistake
            # (tests/test_oracle_mutants.py); otherwise the real one
            lib = ctypes.CDLL(os.environ.get("ORC_LIB") or build())
            d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            pp = ctypes.POINTER(_Params)
            sig = {
                "orc_num_threads": (i, []),
                "orc_set_num_threads": (None, [i]),
                "orc_row_shift": (d, [pp, i]),
                "orc_warp": (None, [pp, vp, vp]),
                "orc_block_stats": (d, [vp, i, i, i, i, i, vp, vp]),
                "orc_ncc": (d, [vp, vp, i, i, i, i, i, i]),
                "orc_bilateral": (d, [vp, i, i, vp, i, i, i, d, d, i, i]),
                "orc_bilateral_slice": (None, [vp, vp, i, i, i, d, d, vp]),
                "orc_wta": (i, [vp, i, vp]),
                "orc_parabola": (d, [vp, i, i, vp]),
                "orc_lr_valid": (i, [i, i, vp, d]),
                "orc_postprocess": (d, [pp, d, i]),
                "orc_reconstruct": (None, [pp, d, i, i, vp, vp, vp]),
                "orc_match": (i, [pp, vp, vp, i, i, ctypes.POINTER(_Outputs)]),
                "orc_match_restricted": (i, [pp, vp, vp, vp, i, i, i, ctypes.POINTER(_Outputs)]),
                "orc_wta_window": (i, [vp, i, i, vp]),
                "orc_match_pixels": (i, [pp, vp, vp, i, vp, vp, vp, vp, vp, vp, vp,
                                         vp, vp, vp]),
                "orc_objective": (d, [pp, vp, vp, vp]),
                "orc_grad": (i, [pp, vp, vp, vp, vp, vp, vp, vp]),
                "orc_fit_alpha": (i, [vp, i, i, i, vp, ctypes.c_float, vp, vp, vp]),
                "orc_fit_roll": (i, [vp, i, i, i, i, i, i, vp, vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Params:
    """Method parameters; names follow the paper (Eqs. 2-12)."""
    W: int
    H: int
    D: int
    ncc_r: int           # block radius of Eq. 3 (n = (2r+1)^2)
    agg_r: int           # bilateral radius rho of Eq. 8
    gamma_d: float       # Eq. 9
    gamma_r: float       # Eq. 10
    lr_thresh: float = 1.0
    alpha0: float = 0.0
    alpha1: float = 0.0
    delta: float = 0.0
    f_px: float = 700.0
    baseline: float = 120.0
    u0: float | None = None
    v0: float | None = None

    def c(self) -> _Params:
        u0 = (self.W - 1) / 2.0 if self.u0 is None else self.u0
        v0 = (self.H - 1) / 2.0 if self.v0 is None else self.v0
        return _Params(self.W, self.H, self.D, self.ncc_r, self.agg_r, self.gamma_d,
                       self.gamma_r, self.lr_thresh, self.alpha0, self.alpha1, self.delta,
                       self.f_px, self.baseline, u0, v0)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    a = np.ascontiguousarray(a)
    assert a.dtype == np.uint8
    return a


def row_shift(p: Params, v: int) -> float:
    return _load().orc_row_shift(ctypes.byref(p.c()), int(v))


def warp(p: Params, right: np.ndarray) -> np.ndarray:
    right = _u8(right)
    out = np.empty((p.H, p.W), np.float64)
    _load().orc_warp(ctypes.byref(p.c()), _ptr(right), _ptr(out))
    return out


def block_stats(img: np.ndarray, r: int, u: int, v: int):
    img = _f64(img)
    H, W = img.shape
    mu, sg = ctypes.c_double(), ctypes.c_double()
    var = _load().orc_block_stats(_ptr(img), W, H, r, u, v, ctypes.byref(mu), ctypes.byref(sg))
    return mu.value, sg.value, var


def ncc(L: np.ndarray, R: np.ndarray, r: int, ul: int, ur: int, v: int) -> float:
    L, R = _f64(L), _f64(R)
    H, W = L.shape
    return _load().orc_ncc(_ptr(L), _ptr(R), W, H, r, ul, ur, v)


def bilateral_slice(slice_: np.ndarray, guide: np.ndarray, rho: int, gamma_d: float,
                    gamma_r: float) -> np.ndarray:
    s, g = _f64(slice_), _f64(guide)
    H, W = s.shape
    out = np.empty_like(s)
    _load().orc_bilateral_slice(_ptr(s), _ptr(g), W, H, rho, gamma_d, gamma_r, _ptr(out))
    return out


def wta(c: np.ndarray):
    c = _f64(c)
    gap = ctypes.c_double()
    best = _load().orc_wta(_ptr(c), c.shape[0], ctypes.byref(gap))
    return best, gap.value


def parabola(c: np.ndarray, d: int):
    c = _f64(c)
    den = ctypes.c_double()
    ds = _load().orc_parabola(_ptr(c), c.shape[0], int(d), ctypes.byref(den))
    return ds, den.value


def lr_valid(u: int, lref: int, ltar_row: np.ndarray, thresh: float) -> bool:
    row = np.ascontiguousarray(ltar_row, dtype=np.int32)
    return bool(_load().orc_lr_valid(int(u), int(lref), _ptr(row), float(thresh)))


def postprocess(p: Params, ds: float, v: int) -> float:
    return _load().orc_postprocess(ctypes.byref(p.c()), float(ds), int(v))


def reconstruct(p: Params, dfull: float, u: int, v: int):
    X, Y, Z = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().orc_reconstruct(ctypes.byref(p.c()), float(dfull), int(u), int(v),
                            ctypes.byref(X), ctypes.byref(Y), ctypes.byref(Z))
    return X.value, Y.value, Z.value


@dataclass
class MatchResult:
    warped: np.ndarray | None = None
    mu_l: np.ndarray | None = None
    sig_l: np.ndarray | None = None
    mu_r: np.ndarray | None = None
    sig_r: np.ndarray | None = None
    cost_l: np.ndarray | None = None
    cost_r: np.ndarray | None = None
    agg_l: np.ndarray | None = None
    agg_r: np.ndarray | None = None
    lbl_l: np.ndarray | None = None
    lbl_r: np.ndarray | None = None
    gap_l: np.ndarray | None = None
    gap_r: np.ndarray | None = None
    den_l: np.ndarray | None = None
    dsub: np.ndarray | None = None
    valid: np.ndarray | None = None
    dfull: np.ndarray | None = None
    xyz: np.ndarray | None = None
    extras: dict = field(default_factory=dict)


_VOLUMES = ("cost_l", "cost_r", "agg_l", "agg_r")


def match(p: Params, left: np.ndarray, right: np.ndarray, rows: tuple[int, int] | None = None,
          want: tuple[str, ...] = ("lbl_l", "lbl_r", "gap_l", "gap_r", "den_l", "dsub",
                                   "valid", "dfull", "xyz"),
          centre: np.ndarray | None = None, radius: int | None = None) -> MatchResult:
    """Run the whole pipeline (or a band of output rows) and return the
    requested arrays.  Unrequested arrays are not computed or stored.  With
    centre ([H, W] residual disparities) and radius, every pixel searches only
    [centre - radius, centre + radius] (clamped to 0..D-1)."""
    left, right = _u8(left), _u8(right)
    assert left.shape == (p.H, p.W) and right.shape == (p.H, p.W)
    H, W, D = p.H, p.W, p.D
    shapes = {
        "warped": ((H, W), np.float64), "mu_l": ((H, W), np.float64),
        "sig_l": ((H, W), np.float64), "mu_r": ((H, W), np.float64),
        "sig_r": ((H, W), np.float64),
        "cost_l": ((H, W, D), np.float64), "cost_r": ((H, W, D), np.float64),
        "agg_l": ((H, W, D), np.float64), "agg_r": ((H, W, D), np.float64),
        "lbl_l": ((H, W), np.int32), "lbl_r": ((H, W), np.int32),
        "gap_l": ((H, W), np.float64), "gap_r": ((H, W), np.float64),
        "den_l": ((H, W), np.float64), "dsub": ((H, W), np.float64),
        "valid": ((H, W), np.uint8), "dfull": ((H, W), np.float64),
        "xyz": ((3, H, W), np.float64),
    }
    res = MatchResult()
    outs = _Outputs()
    for name in want:
        shp, dt = shapes[name]
        fill = np.nan if dt == np.float64 else 0
        arr = np.full(shp, fill, dt)
        setattr(res, name, arr)
        setattr(outs, name, arr.ctypes.data)
    r0, r1 = (0, H) if rows is None else rows
    if centre is None:
        rc = _load().orc_match(ctypes.byref(p.c()), _ptr(left), _ptr(right), int(r0), int(r1),
                               ctypes.byref(outs))
    else:
        c = np.ascontiguousarray(centre, dtype=np.int32)
        assert c.shape == (H, W) and radius is not None
        rc = _load().orc_match_restricted(ctypes.byref(p.c()), _ptr(left), _ptr(right), _ptr(c),
                                          int(radius), int(r0), int(r1), ctypes.byref(outs))
    if rc != 0:
        raise RuntimeError(f"orc_match failed with {rc}")
    return res


def wta_window(c: np.ndarray, lo: int, hi: int):
    """WTA over c[lo..hi] (ties: smallest d); returns (d, gap)."""
    c = _f64(c)
    gap = ctypes.c_double(0.0)
    d = _load().orc_wta_window(_ptr(c), int(lo), int(hi), ctypes.byref(gap))
    return d, gap.value


def match_pixels(p: Params, left: np.ndarray, right: np.ndarray, us, vs) -> dict:
    """The pipeline evaluated independently at sampled pixels."""
    left, right = _u8(left), _u8(right)
    us = np.ascontiguousarray(us, dtype=np.int32)
    vs = np.ascontiguousarray(vs, dtype=np.int32)
    n = us.shape[0]
    out = {
        "lbl_l": np.empty(n, np.int32), "lbl_r_match": np.empty(n, np.int32),
        "gap_l": np.empty(n), "gap_r_match": np.empty(n), "den_l": np.empty(n),
        "dsub": np.empty(n), "valid": np.empty(n, np.uint8), "dfull": np.empty(n),
    }
    rc = _load().orc_match_pixels(
        ctypes.byref(p.c()), _ptr(left), _ptr(right), n, _ptr(us), _ptr(vs),
        _ptr(out["lbl_l"]), _ptr(out["lbl_r_match"]), _ptr(out["gap_l"]),
        _ptr(out["gap_r_match"]), _ptr(out["den_l"]), _ptr(out["dsub"]),
        _ptr(out["valid"]), _ptr(out["dfull"]))
    if rc != 0:
        raise RuntimeError(f"orc_match_pixels failed with {rc}")
    return out


def objective(p: Params, left, right, dstar) -> float:
    """L = sum of the aggregated reference cost at fixed disparities dstar
    (int, -1 = pixel left out); left/right real-valued images."""
    L, R = _f64(left), _f64(right)
    ds = np.ascontiguousarray(dstar, dtype=np.int32)
    return _load().orc_objective(ctypes.byref(p.c()), _ptr(L), _ptr(R), _ptr(ds))


def grad(p: Params, left, right, dstar):
    """(L, dL/dalpha [2], dL/dleft [H,W], dL/dright [H,W]) in FP64."""
    L, R = _f64(left), _f64(right)
    ds = np.ascontiguousarray(dstar, dtype=np.int32)
    out_l = ctypes.c_double()
    da = np.zeros(2)
    gl = np.zeros((p.H, p.W))
    gr = np.zeros((p.H, p.W))
    rc = _load().orc_grad(ctypes.byref(p.c()), _ptr(L), _ptr(R), _ptr(ds), ctypes.byref(out_l),
                          _ptr(da), _ptr(gl), _ptr(gr))
    if rc != 0:
        raise RuntimeError(f"orc_grad failed with {rc}")
    return out_l.value, da, gl, gr


@dataclass
class AlphaFit:
    best: int                 # index of the best hypothesis, -1 if none
    counts: np.ndarray        # inliers per hypothesis, -1 without a model
    alpha: np.ndarray         # least-squares (alpha0, alpha1) through the best's inliers
    n_inliers: int


def fit_alpha(disp: np.ndarray, pairs: np.ndarray, tau: float) -> AlphaFit:
    """Sec. II-A: alpha by least squares with RANSAC over the given point
    pairs (pixel indices v*W+u) of a full-disparity map (NaN = rejected)."""
    d = np.ascontiguousarray(disp, dtype=np.float32)
    H, W = d.shape
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    counts = np.zeros(len(pr), np.int32)
    alpha = np.full(2, np.nan)
    n = ctypes.c_int32(0)
    best = _load().orc_fit_alpha(_ptr(d), W, H, len(pr), _ptr(pr), float(tau), _ptr(counts),
                                 _ptr(alpha), ctypes.byref(n))
    return AlphaFit(best, counts, alpha, n.value)


def fit_roll(disp: np.ndarray, patch: tuple[int, int, int, int]):
    """Sec. II-A roll angle: least-squares plane d = g0 + g1 u + g2 v over the
    valid pixels of patch (u_lo, v_lo, u_hi, v_hi); returns (g[3], roll, n)."""
    d = np.ascontiguousarray(disp, dtype=np.float32)
    H, W = d.shape
    g = np.zeros(3)
    roll = ctypes.c_double(0.0)
    n = _load().orc_fit_roll(_ptr(d), W, H, *[int(x) for x in patch], _ptr(g),
                             ctypes.byref(roll))
    return g, roll.value, n
