"""The near-flat slack used by the parity tests: its block sigma at in-image
centres equals the oracle's sigma of Eq. 5, and it follows the stated form."""
import numpy as np

from helpers import TOL_WARP, near_flat_slack, run_oracle
from paper_1807_07433_gb300 import synth


def test_slack_sigma_equals_oracle_block_sigma():
    w = synth.small(53, 29, D=32, ncc_r=5, agg_r=1, seed=1083)
    left, right, _ = synth.make_pair(w.scene)
    o = run_oracle(w, left, right, ("warped", "sig_r"))
    sl, sr, al, ar = near_flat_slack(o.warped, w.D, w.ncc_r, w.agg_r)
    H, W = left.shape
    clear = (o.sig_r ** 2 > 1.2e-6)
    want = np.minimum(2 * TOL_WARP / np.where(clear, o.sig_r, 1.0), 2.0)
    np.testing.assert_allclose(sr[:, :, 0][clear], want[clear], rtol=1e-9)
    # cost_l at (u, d) takes the warped block at u - d
    for (v, u, d) in ((28, 52, 20), (3, 40, 0), (10, 31, 31)):
        if clear[v, u - d]:
            assert sl[v, u, d] == want[v, u - d]
    # the aggregate's slack covers every cost slack in its window
    assert (al >= sl).all() and (ar >= sr).all()
    assert al[28, 52].max() > 1e-2            # a nearly flat dark patch lies there
