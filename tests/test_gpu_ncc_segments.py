"""The exact-sum NCC kernel at other row-segment lengths (SR_NCC_SEG, read
once per process, so each length runs in a process of its own): one-row
segments, a length that divides nothing, and one segment for the whole
frame.  The costs of both views stay within the cost tolerance of the FP64
oracle (Eq. 3), and bands of the frame still reassemble to the whole frame
bit for bit at every length."""
import os
import subprocess
import sys

import numpy as np
import pytest

from helpers import TOL_COST, run_oracle
from paper_1807_07433_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
W = synth.small(203, 77, D=32, ncc_r=3, agg_r=5, seed=11)

CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
from paper_1807_07433_gb300 import bands, sr, synth
w = synth.small(203, 77, D=32, ncc_r=3, agg_r=5, seed=11)
left, right, _ = synth.make_pair(w.scene)
H, W = left.shape
dl, dr = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
with sr.Matcher(W, H, w.D, w.ncc_r, w.agg_r, w.gamma_d, w.gamma_r, w.lr_thresh,
                stream=torch.cuda.current_stream()) as m:
    m.set_plane(w.scene.alpha0, w.scene.alpha1, w.delta)
    disp = m.match(dl, dr)
    torch.cuda.synchronize()
    full = disp.cpu().numpy()
    cl, cr = m.buffer(sr.SR_BUF_COST_L), m.buffer(sr.SR_BUF_COST_R)
    got = np.full((H, W), -5.0, np.float32)
    for b in bands.plan(H, 3, w.ncc_r, w.agg_r, read_rows=m.band_rows):
        d = m.match_rows(dl[b.r0:b.r1].clone(), dr[b.r0:b.r1].clone(), b.y0, b.y1)
        torch.cuda.synchronize()
        got[b.y0:b.y1] = d.cpu().numpy()
np.savez({out!r}, cost_l=cl, cost_r=cr,
         bands_equal=np.array(np.array_equal(got.view(np.uint32), full.view(np.uint32))))
"""


@pytest.fixture(scope="module")
def oracle_costs():
    left, right, _ = synth.make_pair(W.scene)
    return run_oracle(W, left, right, ("cost_l", "cost_r"))


@pytest.mark.parametrize("seg", [1, 13, 128])
def test_segment_length_keeps_costs_and_bands(seg, oracle_costs, tmp_path):
    out = str(tmp_path / f"seg{seg}.npz")
    env = dict(os.environ, SR_NCC_SEG=str(seg))
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, out=out)], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    z = np.load(out)
    np.testing.assert_allclose(z["cost_l"], oracle_costs.cost_l, rtol=0, atol=TOL_COST)
    np.testing.assert_allclose(z["cost_r"], oracle_costs.cost_r, rtol=0, atol=TOL_COST)
    assert bool(z["bands_equal"])
