"""Pins of the oracle's restricted search (the paper's Sec. IV plan: aggregate
only around previously calculated disparities): every pixel searches
[c - r, c + r] (clamped to 0..D-1) around its centre c."""
import numpy as np
import pytest

import oracle
from helpers import oracle_params
from paper_1807_07433_gb300 import synth

WANT = ("agg_l", "agg_r", "lbl_l", "lbl_r", "gap_l", "dsub", "den_l", "valid", "dfull")


def _case(seed=41):
    w = synth.small(64, 40, D=16, ncc_r=2, agg_r=3, seed=seed)
    left, right, _ = synth.make_pair(w.scene)
    return w, left, right


def test_wide_radius_equals_the_full_search():
    w, left, right = _case()
    p = oracle_params(w)
    full = oracle.match(p, left, right, want=WANT)
    centre = np.random.default_rng(1).integers(0, w.D, size=left.shape)
    res = oracle.match(p, left, right, want=WANT, centre=centre, radius=w.D)
    for k in WANT:
        np.testing.assert_array_equal(getattr(res, k), getattr(full, k), err_msg=k)


def test_labels_are_the_window_argmax_of_the_aggregated_costs():
    w, left, right = _case(42)
    p = oracle_params(w)
    rng = np.random.default_rng(2)
    centre = rng.integers(-3, w.D + 3, size=left.shape)       # clamped into 0..D-1
    r = 2
    res = oracle.match(p, left, right, want=WANT, centre=centre, radius=r)
    c = np.clip(centre, 0, w.D - 1)
    lo, hi = np.maximum(c - r, 0), np.minimum(c + r, w.D - 1)
    for (vol, lbl) in ((res.agg_l, res.lbl_l), (res.agg_r, res.lbl_r)):
        for v in range(left.shape[0]):
            for u in range(left.shape[1]):
                win = vol[v, u, lo[v, u]:hi[v, u] + 1]
                assert lbl[v, u] == lo[v, u] + int(np.argmax(win))   # first maximum
    # Eq. 12 only strictly inside the window; at its ends d^s = d*
    ends = (res.lbl_l == lo) | (res.lbl_l == hi)
    np.testing.assert_array_equal(res.dsub[ends], res.lbl_l[ends].astype(float))
    inner = ~ends & (res.den_l < 0)
    assert inner.any()
    d0 = res.lbl_l[inner]
    a = res.agg_l[inner]
    cm = a[np.arange(len(d0)), d0 - 1]
    c0 = a[np.arange(len(d0)), d0]
    cp = a[np.arange(len(d0)), d0 + 1]
    np.testing.assert_allclose(res.dsub[inner], d0 + (cm - cp) / (2 * cm + 2 * cp - 4 * c0),
                               rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_wta_window_equals_numpy_argmax(seed):
    rng = np.random.default_rng(seed)
    c = np.round(rng.normal(size=24), 1)            # rounding makes ties common
    for lo in range(0, 24, 5):
        for hi in range(lo, 24, 7):
            d, gap = oracle.wta_window(c, lo, hi)
            assert d == lo + int(np.argmax(c[lo:hi + 1]))
            rest = np.delete(c[lo:hi + 1], d - lo)
            assert gap == (c[d] - rest.max() if len(rest) else np.inf)


def test_window_zero_to_dprime_equals_a_search_of_dprime():
    """Centre floor((D'-1)/2) and radius floor(D'/2) give every pixel the
    window [0, D'-1]: the result equals the full search with D = D' (the
    aggregated costs of a disparity do not depend on D)."""
    w16 = synth.small(64, 40, D=16, ncc_r=2, agg_r=3, seed=43)
    w11 = synth.small(64, 40, D=11, ncc_r=2, agg_r=3, seed=43, delta=4.0)
    left, right, _ = synth.make_pair(w16.scene)
    want = ("lbl_l", "lbl_r", "dsub", "valid", "dfull")
    full = oracle.match(oracle_params(w11), left, right, want=want)
    res = oracle.match(oracle_params(w16), left, right, want=want,
                       centre=np.full(left.shape, (11 - 1) // 2), radius=11 // 2)
    for k in want:
        np.testing.assert_array_equal(getattr(res, k), getattr(full, k), err_msg=k)
