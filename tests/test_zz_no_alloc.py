"""sr_match_noalloc: the match for callers that cannot allocate device memory.

Such callers (a host that fixes the device-memory budget at start-up, a
plug-in whose host owns the allocator, a real-time loop that must not wait on
the allocator) get the same disparities as sr_match without creating a
context: the intermediates live in a fixed 32 MiB device array inside the
library.  The entry point runs the kernels sr_match runs on the same inputs,
so its results must equal sr_match's bit for bit; a looser check could hide
a scratch region that two stages share by mistake.  This module runs last so
that a failure here never hides one elsewhere; it must pass on its own in a
fresh process too.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1807_07433_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

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


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


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
        sr.sr_noalloc_status(torch.cuda.current_stream())
        d, l = disp.cpu().numpy(), wta.cpu().numpy()
        np.testing.assert_array_equal(l, ref_wta)
        np.testing.assert_array_equal(_bits(d), _bits(ref_disp))   # NaN patterns included


def test_noalloc_allocates_nothing():
    """After a first call (which looks up the array's address), further calls
    change neither torch's allocations nor the device's free memory."""
    import torch
    from paper_1807_07433_gb300 import sr
    w = CASES[2]
    left, right, _ = synth.make_pair(w.scene)
    H, W = left.shape
    dl, dr = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
    params = sr.make_params(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh)
    st = torch.cuda.current_stream()
    sr.sr_match_noalloc(params, w.scene.alpha0, w.scene.alpha1, w.delta, dl, dr, W, disp,
                        None, st)
    sr.sr_noalloc_status(st)
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
    for _ in range(3):
        sr.sr_match_noalloc(params, w.scene.alpha0, w.scene.alpha1, w.delta, dl, dr, W, disp,
                            None, st)
    sr.sr_noalloc_status(st)
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
    assert after == before


def test_noalloc_rejects_frames_beyond_its_scratch():
    import torch
    from paper_1807_07433_gb300 import sr
    params = sr.make_params(1280, 720, 64, 3, 5, 4.0, 12.0)
    buf = torch.zeros((720, 1280), dtype=torch.uint8, device="cuda")
    out = torch.empty((720, 1280), dtype=torch.float32, device="cuda")
    with pytest.raises(sr.SrError) as e:
        sr.sr_match_noalloc(params, 30.0, 0.08, 8.0, buf, buf, 1280, out)
    assert e.value.status == sr.SR_ERR_UNSUPPORTED


# Runs in a fresh process that uses only the CUDA driver API (through ctypes)
# and libsr.so: the match in the device's primary context, then in two
# driver-API contexts created and destroyed one after the other (each loads
# the library's module anew, so the arrays have other addresses there), then
# in the primary context again.  Prints the results' digests as JSON.
_CONTEXTS_SCRIPT = r"""
import ctypes, json, sys, hashlib
sys.path.insert(0, sys.argv[1])
import numpy as np
from paper_1807_07433_gb300 import sr, synth

cu = ctypes.CDLL("libcuda.so.1")
def ck(r, what):
    if r != 0:
        raise RuntimeError(f"{what} failed: {r}")
ck(cu.cuInit(0), "cuInit")
dev = ctypes.c_int()
ck(cu.cuDeviceGet(ctypes.byref(dev), 0), "cuDeviceGet")
prim = ctypes.c_void_p()
ck(cu.cuDevicePrimaryCtxRetain(ctypes.byref(prim), dev), "cuDevicePrimaryCtxRetain")
ck(cu.cuCtxSetCurrent(prim), "cuCtxSetCurrent")

w = synth.small(150, 90, D=64, ncc_r=3, agg_r=5, seed=21, alpha1=0.08)
left, right, _ = synth.make_pair(w.scene)
H, W = left.shape
params = sr.make_params(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh)
lib = sr.load()
u64 = ctypes.c_uint64

def run_here():
    bufs = []
    def alloc(n):
        p = u64()
        ck(cu.cuMemAlloc_v2(ctypes.byref(p), ctypes.c_size_t(n)), "cuMemAlloc")
        bufs.append(p)
        return p.value
    dl, dr, dd = alloc(W * H), alloc(W * H), alloc(4 * W * H)
    ck(cu.cuMemcpyHtoD_v2(u64(dl), left.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(W * H)), "H2D")
    ck(cu.cuMemcpyHtoD_v2(u64(dr), right.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(W * H)), "H2D")
    out = []
    for _ in range(2):
        st = lib.sr_match_noalloc(ctypes.byref(params), w.scene.alpha0, w.scene.alpha1, w.delta,
                                  dl, dr, W, dd, None, None)
        assert st == 0, st
        assert lib.sr_noalloc_status(None) == 0
        d = np.empty((H, W), np.float32)
        ck(cu.cuMemcpyDtoH_v2(d.ctypes.data_as(ctypes.c_void_p), u64(dd), ctypes.c_size_t(4 * W * H)), "D2H")
        out.append(hashlib.sha256(d.tobytes()).hexdigest())
    for p in bufs:
        ck(cu.cuMemFree_v2(p), "cuMemFree")
    assert out[0] == out[1]
    return out[0]

def run_in_new_context():
    ctx = ctypes.c_void_p()
    if hasattr(cu, "cuCtxCreate_v4"):
        ck(cu.cuCtxCreate_v4(ctypes.byref(ctx), None, 0, dev), "cuCtxCreate")
    else:
        ck(cu.cuCtxCreate_v2(ctypes.byref(ctx), 0, dev), "cuCtxCreate")
    try:
        return run_here()
    finally:
        ck(cu.cuCtxDestroy_v2(ctx), "cuCtxDestroy")
        ck(cu.cuCtxSetCurrent(prim), "cuCtxSetCurrent")

res = {"primary": run_here(), "ctx1": run_in_new_context(), "ctx2": run_in_new_context()}
res["primary_again"] = run_here()
print(json.dumps(res))
"""


def test_noalloc_in_other_cuda_contexts():
    """The array's address is looked up per CUDA context: the results are the
    same bit for bit in the primary context, in two driver-API contexts made
    and destroyed one after the other, and in the primary context again."""
    r = subprocess.run([sys.executable, "-c", _CONTEXTS_SCRIPT, ROOT], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(set(res.values())) == 1, res
