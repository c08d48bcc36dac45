"""Bounds-checked build (SR_BOUNDS_CHECK, libsr_check.so) on the GPU.

The checked library runs the match path -- the stage-parity scenes (ragged,
tiny and degenerate sizes), the 1280x720x64 frame at FP32 and FP16, the
restricted search, row bands, reconstruction, and a mixed-size batch under
the persistent, per-pair and sr_match-kernel schedules -- in a child
process. Every checked index stays inside its buffer (sr_bounds_report:
SR_OK after each case), and every output equals the release library's bit
for bit (the checks change no arithmetic). A self-test flag makes the
checked reconstruction record one offence without any memory access: the
call returns SR_ERR_BOUNDS, the report gives its site and index, and the
context works on.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked(tmp_path_factory):
    from paper_1807_07433_gb300 import _build
    _build.build(check=True)
    out = str(tmp_path_factory.mktemp("bounds") / "checked.npz")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_child.py"), out],
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(out))


def test_no_index_out_of_range(checked):
    from paper_1807_07433_gb300 import sr
    import bounds_child
    for name, _, _ in bounds_child.CASES:
        st, site, index, count = checked[f"{name}.report"]
        assert st == sr.SR_OK and count == 0, (name, site, index, count)


def test_outputs_equal_release_build(checked):
    """Release library in this process, same cases: identical arrays."""
    import bounds_child
    ran = 0
    for name, w, vt in bounds_child.CASES:
        ref = bounds_child.run_case(w, vt)
        for k, v in ref.items():
            got = checked[f"{name}.{k}"]
            assert got.shape == v.shape, (name, k)
            assert np.array_equal(got.view(np.uint8), v.view(np.uint8)), (name, k)
            ran += 1
    assert ran >= 3 * len(bounds_child.CASES)


def test_batch_schedules_in_range_and_equal(checked):
    """The persistent, descriptor-driven and per-pair batch schedules: no
    offence, and the same outputs as the release library's."""
    from paper_1807_07433_gb300 import sr
    import bounds_child
    for v in bounds_child.BATCH_VARIANTS:
        st, site, index, count = checked[f"batch{v}.report"]
        assert st == sr.SR_OK and count == 0, (v, site, index, count)
        ref = bounds_child.run_batch(v)
        for k, a in ref.items():
            assert np.array_equal(checked[f"batch{v}.{k}"].view(np.uint8), a.view(np.uint8)), (v, k)


def test_selftest_reports_through_the_abi(checked):
    from paper_1807_07433_gb300 import sr
    assert int(checked["selftest.call_status"]) == sr.SR_ERR_BOUNDS
    st, site, index, count = checked["selftest.report"]
    assert (st, site, index, count) == (sr.SR_ERR_BOUNDS, 399, -1, 1)
    assert "k_pixel" in str(checked["selftest.unit"])
    st, site, index, count = checked["after.report"]
    assert st == sr.SR_OK and count == 0


def test_release_build_reports_unsupported():
    from paper_1807_07433_gb300 import sr
    assert sr.sr_bounds_report()[0] == sr.SR_ERR_UNSUPPORTED
