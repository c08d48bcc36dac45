"""Precision form: cost volumes stored in FP16 / BF16, FP32 arithmetic.

Bounds follow from the storage rounding alone.  A cost c in [-1, 1] rounded
to a format with p significand bits moves by at most 2^-p (FP16: p = 11,
BF16: p = 8); the FP32 path adds at most TOL_COST.  The aggregated cost is a
weighted mean of stored costs, so it moves by at most the same eps.  A label
can then differ only where the oracle's top-2 gap is below 2 eps, and the
Eq. 12 offset by at most 6 eps / |den| (numerator error 2 eps, denominator
8 eps times an offset <= 1/2).
"""
import numpy as np
import pytest

from helpers import TOL_COST, oracle_params, run_gpu, run_oracle
from paper_1807_07433_gb300 import synth

pytestmark = pytest.mark.gpu

EPS = {"f16": 2.0 ** -11 + TOL_COST, "bf16": 2.0 ** -8 + TOL_COST}
WANT = ("cost_l", "cost_r", "agg_l", "agg_r", "lbl_l", "lbl_r", "gap_l", "gap_r", "den_l",
        "dsub", "valid", "dfull")
CASES = [synth.C1, synth.small(203, 77, D=32, ncc_r=3, agg_r=5, seed=11),
         synth.small(131, 64, D=64, ncc_r=3, agg_r=5, seed=31, alpha1=0.08)]


def _buffers(sr):
    return (("cost_l", sr.SR_BUF_COST_L), ("cost_r", sr.SR_BUF_COST_R),
            ("agg_l", sr.SR_BUF_AGG_L), ("agg_r", sr.SR_BUF_AGG_R),
            ("lbl_l", sr.SR_BUF_WTA_L), ("lbl_r", sr.SR_BUF_WTA_R), ("dsub", sr.SR_BUF_DSUB))


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_low_precision_volumes_within_rounding_bounds(w, dtype):
    from paper_1807_07433_gb300 import sr
    vt = {"f16": sr.SR_VOL_F16, "bf16": sr.SR_VOL_BF16}[dtype]
    eps = EPS[dtype]
    left, right, _ = synth.make_pair(w.scene)
    g = run_gpu(w, left, right, keep_agg=True, buffers=_buffers(sr), vol_dtype=vt)
    o = run_oracle(w, left, right, WANT)
    np.testing.assert_allclose(g["cost_l"], o.cost_l, rtol=0, atol=eps)
    np.testing.assert_allclose(g["cost_r"], o.cost_r, rtol=0, atol=eps)
    np.testing.assert_allclose(g["agg_l"], o.agg_l, rtol=0, atol=eps)
    np.testing.assert_allclose(g["agg_r"], o.agg_r, rtol=0, atol=eps)
    for side in ("l", "r"):
        diff = g["lbl_" + side] != getattr(o, "lbl_" + side)
        assert np.all(getattr(o, "gap_" + side)[diff] < 2 * eps)
    same = (g["lbl_l"] == o.lbl_l) & (o.gap_l >= 2 * eps) & (o.den_l != 0.0)
    bound = 6 * eps / np.abs(o.den_l[same])
    assert np.all(np.abs(g["dsub"][same] - o.dsub[same]) <= bound + 1e-6)


def test_fp16_and_bf16_rank_as_expected_at_full_size():
    """1280x720x64: the 16-bit forms agree with the FP32 form on almost all
    labels, BF16 (8-bit significand) no better than FP16 (11-bit)."""
    from paper_1807_07433_gb300 import sr
    w = synth.C2
    left, right, _ = synth.make_pair(w.scene)
    res = {vt: run_gpu(w, left, right, vol_dtype=vt)
           for vt in (sr.SR_VOL_F32, sr.SR_VOL_F16, sr.SR_VOL_BF16)}
    ref = res[sr.SR_VOL_F32]["wta"]
    m16 = np.mean(res[sr.SR_VOL_F16]["wta"] != ref)
    mbf = np.mean(res[sr.SR_VOL_BF16]["wta"] != ref)
    assert m16 <= 0.01 and mbf <= 0.05
    assert m16 <= mbf
