"""Python binding of the C ABI in include/sr.h (ctypes; argument marshalling only).

Every function keeps the C name and order of arguments.  Device buffers are
passed as torch CUDA tensors (or raw integer device pointers); all arithmetic
runs in libsr.so's CUDA kernels.  If libsr.so is missing this module raises on
first use -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsr.so")
CHECK_LIB_PATH = os.path.join(_HERE, "libsr_check.so")   # bounds-checked build

SR_OK, SR_ERR_INVALID_ARG, SR_ERR_UNSUPPORTED, SR_ERR_OOM, SR_ERR_CUDA, SR_ERR_STATE, \
    SR_ERR_TIMEOUT, SR_ERR_BOUNDS = range(8)
SR_VOL_F32, SR_VOL_F16, SR_VOL_BF16 = range(3)
(SR_BUF_WARPED, SR_BUF_MU_L, SR_BUF_INV_L, SR_BUF_MU_R, SR_BUF_INV_R, SR_BUF_COST_L,
 SR_BUF_COST_R, SR_BUF_AGG_L, SR_BUF_AGG_R, SR_BUF_WTA_L, SR_BUF_WTA_R, SR_BUF_DSUB) = range(12)
SR_DEBUG_KEEP_AGG = 1
SR_DEBUG_WITHHOLD_ROW = 2
SR_DEBUG_NO_BAND = 4
SR_DEBUG_BOUNDS_SELFTEST = 8

# Functions the header declares (tests check the library exports each one).
EXPORTS = ("sr_create", "sr_destroy", "sr_set_plane", "sr_set_camera", "sr_match",
           "sr_match_restricted", "sr_match_rows", "sr_band_rows",
           "sr_match_host", "sr_match_host_async", "sr_match_noalloc", "sr_noalloc_status",
           "sr_bounds_report",
           "sr_match_batch", "sr_set_autotune",
           "sr_set_batch_schedule", "sr_batch_info", "sr_reconstruct", "sr_grad_plane",
           "sr_fit_alpha", "sr_fit_roll",
           "sr_get_buffer", "sr_set_debug",
           "sr_set_profiling", "sr_synchronize", "sr_stage_times", "sr_stage_times_history", "sr_stage_names", "sr_kernels_per_match",
           "sr_status_str", "sr_last_error", "sr_version")


class sr_params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("max_disp", ctypes.c_int),
                ("ncc_radius", ctypes.c_int), ("agg_radius", ctypes.c_int),
                ("gamma_d", ctypes.c_float), ("gamma_r", ctypes.c_float),
                ("lr_thresh", ctypes.c_float), ("vol_dtype", ctypes.c_int)]


class sr_pair_desc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int),
                ("pitch_bytes", ctypes.c_int), ("d_left", ctypes.c_void_p),
                ("d_right", ctypes.c_void_p), ("alpha0", ctypes.c_double),
                ("alpha1", ctypes.c_double), ("delta", ctypes.c_double),
                ("d_disp", ctypes.c_void_p), ("d_wta_or_null", ctypes.c_void_p)]


class SrError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {status_name(status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libsr.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise OSError(f"{p} not found: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(p)
            vp, i, d, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_float
            sz = ctypes.c_size_t
            sigs = {
                "sr_create": (i, [ctypes.POINTER(sr_params), vp, ctypes.POINTER(vp)]),
                "sr_destroy": (i, [vp]),
                "sr_set_plane": (i, [vp, d, d, d]),
                "sr_set_camera": (i, [vp, d, d, d, d]),
                "sr_match": (i, [vp, vp, vp, i, vp, vp]),
                "sr_match_host": (i, [vp, vp, vp, vp]),
                "sr_match_host_async": (i, [vp, vp, vp, vp]),
                "sr_match_restricted": (i, [vp, vp, vp, i, vp, i, vp, vp]),
                "sr_match_rows": (i, [vp, vp, vp, i, i, i, vp, vp]),
                "sr_band_rows": (i, [vp, i, i, ctypes.POINTER(i), ctypes.POINTER(i)]),
                "sr_match_noalloc": (i, [ctypes.POINTER(sr_params), d, d, d, vp, vp, i, vp, vp,
                                         vp]),
                "sr_noalloc_status": (i, [vp]),
                "sr_bounds_report": (i, [ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.c_char_p, i, ctypes.POINTER(ctypes.c_longlong)]),
                "sr_match_batch": (i, [vp, i, ctypes.POINTER(sr_pair_desc)]),
                "sr_set_autotune": (i, [vp, i, ctypes.c_char_p]),
                "sr_batch_info": (i, [vp, ctypes.c_char_p, sz]),
                "sr_set_batch_schedule": (i, [vp, i]),
                "sr_reconstruct": (i, [vp, vp, vp]),
                "sr_grad_plane": (i, [vp, vp, vp, i, vp, ctypes.POINTER(d), vp, vp]),
                "sr_fit_alpha": (i, [vp, vp, i, vp, f, ctypes.POINTER(d), vp,
                                     ctypes.POINTER(i), ctypes.POINTER(i)]),
                "sr_fit_roll": (i, [vp, vp, i, i, i, i, ctypes.POINTER(d), ctypes.POINTER(d),
                                    ctypes.POINTER(i)]),
                "sr_get_buffer": (i, [vp, i, vp, ctypes.POINTER(sz)]),
                "sr_set_debug": (i, [vp, i]),
                "sr_set_profiling": (i, [vp, i]),
                "sr_synchronize": (i, [vp]),
                "sr_stage_times": (i, [vp, ctypes.POINTER(f), i, ctypes.POINTER(i)]),
                "sr_stage_times_history": (i, [vp, ctypes.POINTER(f), i, ctypes.POINTER(i)]),
                "sr_stage_names": (ctypes.c_char_p, []),
                "sr_kernels_per_match": (i, [vp]),
                "sr_status_str": (ctypes.c_char_p, [i]),
                "sr_last_error": (ctypes.c_char_p, [vp]),
                "sr_version": (ctypes.c_char_p, []),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_name(s: int) -> str:
    try:
        return load().sr_status_str(int(s)).decode()
    except OSError:
        return f"status {s}"


def _ptr(x) -> int | None:
    """Device/host address of a torch tensor, numpy array or raw int (None = NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _check(ctx, status: int, where: str):
    if status != SR_OK:
        detail = load().sr_last_error(ctx).decode() if ctx else ""
        raise SrError(status, where, detail)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(width, height, max_disp, ncc_radius, agg_radius, gamma_d, gamma_r,
                lr_thresh=1.0, vol_dtype=SR_VOL_F32) -> sr_params:
    return sr_params(int(width), int(height), int(max_disp), int(ncc_radius), int(agg_radius),
                     float(gamma_d), float(gamma_r), float(lr_thresh), int(vol_dtype))


def sr_create(params: sr_params, cuda_stream=None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(None, load().sr_create(ctypes.byref(params), _stream_handle(cuda_stream),
                                  ctypes.byref(ctx)), "sr_create")
    return ctx


def sr_destroy(ctx) -> None:
    _check(None, load().sr_destroy(ctx), "sr_destroy")


def sr_set_plane(ctx, alpha0: float, alpha1: float, delta: float) -> None:
    _check(ctx, load().sr_set_plane(ctx, alpha0, alpha1, delta), "sr_set_plane")


def sr_set_camera(ctx, f_px: float, baseline: float, u0: float, v0: float) -> None:
    _check(ctx, load().sr_set_camera(ctx, f_px, baseline, u0, v0), "sr_set_camera")


def sr_match(ctx, d_left, d_right, pitch_bytes: int, d_disp, d_wta_or_null=None) -> None:
    _check(ctx, load().sr_match(ctx, _ptr(d_left), _ptr(d_right), int(pitch_bytes),
                                _ptr(d_disp), _ptr(d_wta_or_null)), "sr_match")


def sr_match_restricted(ctx, d_left, d_right, pitch_bytes: int, d_centre, radius: int, d_disp,
                        d_wta_or_null=None) -> None:
    _check(ctx, load().sr_match_restricted(ctx, _ptr(d_left), _ptr(d_right), int(pitch_bytes),
                                           _ptr(d_centre), int(radius), _ptr(d_disp),
                                           _ptr(d_wta_or_null)), "sr_match_restricted")


def sr_match_rows(ctx, d_left_rows, d_right_rows, pitch_bytes: int, y0: int, y1: int,
                  d_disp_rows, d_wta_rows_or_null=None) -> None:
    _check(ctx, load().sr_match_rows(ctx, _ptr(d_left_rows), _ptr(d_right_rows),
                                     int(pitch_bytes), int(y0), int(y1), _ptr(d_disp_rows),
                                     _ptr(d_wta_rows_or_null)), "sr_match_rows")


def sr_band_rows(ctx, y0: int, y1: int) -> tuple[int, int]:
    """Image rows [r0, r1) that sr_match_rows reads for output rows [y0, y1)."""
    r0, r1 = ctypes.c_int(0), ctypes.c_int(0)
    _check(ctx, load().sr_band_rows(ctx, int(y0), int(y1), ctypes.byref(r0), ctypes.byref(r1)),
           "sr_band_rows")
    return r0.value, r1.value


def sr_match_host(ctx, h_left, h_right, h_disp) -> None:
    _check(ctx, load().sr_match_host(ctx, _ptr(h_left), _ptr(h_right), _ptr(h_disp)),
           "sr_match_host")


def sr_match_host_async(ctx, h_left, h_right, h_disp) -> None:
    """Queue one frame of host buffers (see sr.h); sr_synchronize finishes it."""
    _check(ctx, load().sr_match_host_async(ctx, _ptr(h_left), _ptr(h_right), _ptr(h_disp)),
           "sr_match_host_async")


def sr_match_noalloc(params: sr_params, alpha0: float, alpha1: float, delta: float, d_left,
                     d_right, pitch_bytes: int, d_disp, d_wta_or_null=None,
                     cuda_stream=None) -> None:
    """sr_match without a context and without any device allocation, for
    callers that may not allocate (see include/sr.h for the size limit)."""
    _check(None, load().sr_match_noalloc(ctypes.byref(params), alpha0, alpha1, delta,
                                         _ptr(d_left), _ptr(d_right), int(pitch_bytes),
                                         _ptr(d_disp), _ptr(d_wta_or_null),
                                         _stream_handle(cuda_stream)), "sr_match_noalloc")


def sr_noalloc_status(cuda_stream=None) -> None:
    """Synchronise the stream; raise SrError(SR_ERR_TIMEOUT) if a bounded wait
    of an sr_match_noalloc call in the current context ran out since the last
    check (the condition is then cleared)."""
    _check(None, load().sr_noalloc_status(_stream_handle(cuda_stream)), "sr_noalloc_status")


def sr_bounds_report():
    """Bounds-checked build: (status, site, index, unit, count) of the first
    out-of-range index recorded since the last report (status SR_OK: none,
    SR_ERR_BOUNDS: one; SR_ERR_UNSUPPORTED in a release build); clears it."""
    site, index, count = ctypes.c_int(-1), ctypes.c_longlong(0), ctypes.c_longlong(0)
    unit = ctypes.create_string_buffer(160)
    st = load().sr_bounds_report(ctypes.byref(site), ctypes.byref(index), unit, 160,
                                 ctypes.byref(count))
    return st, site.value, index.value, unit.value.decode(errors="replace"), count.value


def make_pair_desc(left, right, disp, alpha0, alpha1, delta, wta=None) -> sr_pair_desc:
    """Descriptor of one pair (torch CUDA tensors [H, W])."""
    H, W = left.shape
    return sr_pair_desc(int(W), int(H), int(left.stride(0) * left.element_size()), _ptr(left),
                        _ptr(right), float(alpha0), float(alpha1), float(delta), _ptr(disp),
                        _ptr(wta))


def sr_match_batch(ctx, pairs) -> None:
    arr = (sr_pair_desc * len(pairs))(*pairs)
    _check(ctx, load().sr_match_batch(ctx, len(pairs), arr), "sr_match_batch")


def sr_set_autotune(ctx, enable: bool, cache_path: str | None = None) -> None:
    _check(ctx, load().sr_set_autotune(ctx, int(bool(enable)),
                                       cache_path.encode() if cache_path else None),
           "sr_set_autotune")


def sr_set_batch_schedule(ctx, variant: int) -> None:
    _check(ctx, load().sr_set_batch_schedule(ctx, int(variant)), "sr_set_batch_schedule")


def sr_batch_info(ctx) -> dict:
    import json
    buf = ctypes.create_string_buffer(1024)
    _check(ctx, load().sr_batch_info(ctx, buf, 1024), "sr_batch_info")
    return json.loads(buf.value.decode())


def sr_reconstruct(ctx, d_disp, d_xyz) -> None:
    _check(ctx, load().sr_reconstruct(ctx, _ptr(d_disp), _ptr(d_xyz)), "sr_reconstruct")


def sr_grad_plane(ctx, d_left, d_right, pitch_bytes: int, d_dstar, d_grad_left=None,
                  d_grad_right=None) -> np.ndarray:
    """Returns [L, dL/dalpha0, dL/dalpha1]; fills the optional image gradients."""
    out = (ctypes.c_double * 3)()
    _check(ctx, load().sr_grad_plane(ctx, _ptr(d_left), _ptr(d_right), int(pitch_bytes),
                                     _ptr(d_dstar), out, _ptr(d_grad_left), _ptr(d_grad_right)),
           "sr_grad_plane")
    return np.array(out[:], np.float64)


def sr_fit_alpha(ctx, d_disp, pairs, tau_px: float) -> dict:
    """RANSAC + least squares for alpha of Eq. 2; pairs: int [n, 2] pixel indices."""
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    alpha = (ctypes.c_double * 2)()
    counts = np.zeros(len(pr), np.int32)
    best, n_in = ctypes.c_int(-1), ctypes.c_int(0)
    _check(ctx, load().sr_fit_alpha(ctx, _ptr(d_disp), len(pr), pr.ctypes.data, float(tau_px),
                                    alpha, counts.ctypes.data, ctypes.byref(best),
                                    ctypes.byref(n_in)), "sr_fit_alpha")
    return {"alpha": np.array(alpha[:]), "counts": counts, "best": best.value,
            "n_inliers": n_in.value}


def sr_fit_roll(ctx, d_disp, u_lo: int, v_lo: int, u_hi: int, v_hi: int):
    """Plane d = g0 + g1 u + g2 v over a patch; returns (g[3], roll, n)."""
    g = (ctypes.c_double * 3)()
    roll, n = ctypes.c_double(0.0), ctypes.c_int(0)
    _check(ctx, load().sr_fit_roll(ctx, _ptr(d_disp), int(u_lo), int(v_lo), int(u_hi), int(v_hi),
                                   g, ctypes.byref(roll), ctypes.byref(n)), "sr_fit_roll")
    return np.array(g[:]), roll.value, n.value


def sr_get_buffer(ctx, which: int, dst, nbytes: int) -> int:
    n = ctypes.c_size_t(nbytes)
    _check(ctx, load().sr_get_buffer(ctx, int(which), _ptr(dst), ctypes.byref(n)),
           "sr_get_buffer")
    return n.value


def sr_set_debug(ctx, flags: int) -> None:
    _check(ctx, load().sr_set_debug(ctx, int(flags)), "sr_set_debug")


def sr_set_profiling(ctx, enable: bool) -> None:
    _check(ctx, load().sr_set_profiling(ctx, int(bool(enable))), "sr_set_profiling")


def sr_synchronize(ctx) -> None:
    _check(ctx, load().sr_synchronize(ctx), "sr_synchronize")


def sr_stage_times(ctx) -> dict:
    n = 16
    arr = (ctypes.c_float * n)()
    cnt = ctypes.c_int()
    _check(ctx, load().sr_stage_times(ctx, arr, n, ctypes.byref(cnt)), "sr_stage_times")
    names = sr_stage_names()
    return {names[k]: float(arr[k]) for k in range(cnt.value)}


def sr_stage_times_history(ctx, max_matches: int) -> list[dict]:
    """Stage durations (ms) of the most recent matches recorded while
    profiling, oldest first (at most 512)."""
    names = sr_stage_names()
    arr = (ctypes.c_float * (int(max_matches) * len(names)))()
    cnt = ctypes.c_int()
    _check(ctx, load().sr_stage_times_history(ctx, arr, int(max_matches), ctypes.byref(cnt)),
           "sr_stage_times_history")
    return [{names[s]: float(arr[k * len(names) + s]) for s in range(len(names))}
            for k in range(cnt.value)]


def sr_stage_names() -> list[str]:
    return load().sr_stage_names().decode().split(",")


def sr_kernels_per_match(ctx) -> int:
    return int(load().sr_kernels_per_match(ctx))


def sr_version() -> str:
    return load().sr_version().decode()


# ------------------------------------------------------------ convenience layer

_BUF_SPEC = {  # which -> (dtype, per-pixel shape suffix uses D?)
    SR_BUF_WARPED: (np.float32, False), SR_BUF_MU_L: (np.float32, False),
    SR_BUF_INV_L: (np.float32, False), SR_BUF_MU_R: (np.float32, False),
    SR_BUF_INV_R: (np.float32, False), SR_BUF_COST_L: (np.float32, True),
    SR_BUF_COST_R: (np.float32, True), SR_BUF_AGG_L: (np.float32, True),
    SR_BUF_AGG_R: (np.float32, True), SR_BUF_WTA_L: (np.int16, False),
    SR_BUF_WTA_R: (np.int16, False), SR_BUF_DSUB: (np.float32, False),
}


class Matcher:
    """A context plus the calls a user makes, on torch tensors.

    >>> m = Matcher(W, H, D, ncc_radius, agg_radius, gamma_d, gamma_r)
    >>> m.set_plane(alpha0, alpha1, delta)
    >>> disp = m.match(left_u8_cuda, right_u8_cuda)       # float32 [H, W], NaN = rejected
    """

    def __init__(self, width, height, max_disp, ncc_radius, agg_radius, gamma_d, gamma_r,
                 lr_thresh=1.0, vol_dtype=SR_VOL_F32, stream=None):
        self.params = make_params(width, height, max_disp, ncc_radius, agg_radius, gamma_d,
                                  gamma_r, lr_thresh, vol_dtype)
        self.W, self.H, self.D = int(width), int(height), int(max_disp)
        self.ctx = sr_create(self.params, stream)

    def close(self):
        if self.ctx is not None:
            sr_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_plane(self, alpha0, alpha1, delta):
        sr_set_plane(self.ctx, alpha0, alpha1, delta)

    def set_camera(self, f_px, baseline, u0=None, v0=None):
        u0 = (self.W - 1) / 2.0 if u0 is None else u0
        v0 = (self.H - 1) / 2.0 if v0 is None else v0
        sr_set_camera(self.ctx, f_px, baseline, u0, v0)

    def match(self, left, right, disp=None, wta=None):
        import torch
        if disp is None:
            disp = torch.empty((self.H, self.W), dtype=torch.float32, device=left.device)
        pitch = left.stride(0) * left.element_size()
        assert right.stride(0) == left.stride(0), "left and right must share a pitch"
        sr_match(self.ctx, left, right, pitch, disp, wta)
        return disp

    def match_restricted(self, left, right, radius, centre=None, disp=None, wta=None):
        """sr_match_restricted: search [centre - radius, centre + radius] per
        pixel (centre: int16 [H, W] CUDA tensor, None = round(delta))."""
        import torch
        if disp is None:
            disp = torch.empty((self.H, self.W), dtype=torch.float32, device=left.device)
        pitch = left.stride(0) * left.element_size()
        assert right.stride(0) == left.stride(0), "left and right must share a pitch"
        if centre is not None:
            assert centre.dtype == torch.int16 and centre.is_contiguous()
        sr_match_restricted(self.ctx, left, right, pitch, centre, radius, disp, wta)
        return disp

    def band_rows(self, y0, y1):
        """sr_band_rows: the image rows (r0, r1) that match_rows reads for
        output rows [y0, y1)."""
        return sr_band_rows(self.ctx, y0, y1)

    def match_rows(self, left_rows, right_rows, y0, y1, disp_rows=None, wta_rows=None):
        """sr_match_rows: rows [y0, y1) of the frame's disparity map from the
        image rows r0..r1-1 (band plus halo, band_rows; see bands.plan) given
        as [r1 - r0, W] CUDA tensors."""
        import torch
        if disp_rows is None:
            disp_rows = torch.empty((y1 - y0, self.W), dtype=torch.float32,
                                    device=left_rows.device)
        pitch = left_rows.stride(0) * left_rows.element_size()
        assert right_rows.stride(0) == left_rows.stride(0), "left and right must share a pitch"
        sr_match_rows(self.ctx, left_rows, right_rows, pitch, y0, y1, disp_rows, wta_rows)
        return disp_rows

    def reconstruct(self, disp, xyz=None):
        import torch
        if xyz is None:
            xyz = torch.empty((3, self.H, self.W), dtype=torch.float32, device=disp.device)
        sr_reconstruct(self.ctx, disp, xyz)
        return xyz

    def grad_plane(self, left, right, dstar, image_grads=False):
        """L and dL/dalpha of the aggregated cost at fixed disparities dstar
        (int16 [H, W] CUDA tensor, -1 = left out), at the current plane.
        Returns (L, dL/dalpha [2]) or, with image_grads, also dL/di_l and
        dL/di_r as float32 [H, W] CUDA tensors."""
        import torch
        assert dstar.dtype == torch.int16 and dstar.is_contiguous()
        pitch = left.stride(0) * left.element_size()
        assert right.stride(0) == left.stride(0), "left and right must share a pitch"
        gl = gr = None
        if image_grads:
            gl = torch.empty((self.H, self.W), dtype=torch.float32, device=left.device)
            gr = torch.empty_like(gl)
        out = sr_grad_plane(self.ctx, left, right, pitch, dstar, gl, gr)
        if image_grads:
            return float(out[0]), out[1:].copy(), gl, gr
        return float(out[0]), out[1:].copy()

    def buffer(self, which: int) -> np.ndarray:
        dt, vol = _BUF_SPEC[which]
        shape = (self.H, self.W, self.D) if vol else (self.H, self.W)
        out = np.empty(shape, dt)
        sr_get_buffer(self.ctx, which, out, out.nbytes)
        return out
