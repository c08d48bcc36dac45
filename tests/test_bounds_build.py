"""Host-side checks of the bounds-checked build (no GPU): the status code
agrees between the header and the binding, the release library answers the
report call with SR_ERR_UNSUPPORTED without touching the device, and a
kernel file compiles with SR_BOUNDS_CHECK for sm_103a."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_status_code_matches_header():
    from paper_1807_07433_gb300 import sr
    h = open(os.path.join(ROOT, "include", "sr.h")).read()
    m = re.search(r"SR_ERR_BOUNDS\s*=\s*(\d+)", h)
    assert m and int(m.group(1)) == sr.SR_ERR_BOUNDS
    m = re.search(r"#define SR_DEBUG_BOUNDS_SELFTEST\s+(\d+)", h)
    assert m and int(m.group(1)) == sr.SR_DEBUG_BOUNDS_SELFTEST


def test_release_library_reports_unsupported():
    from paper_1807_07433_gb300 import sr
    if not os.path.exists(sr.LIB_PATH):
        pytest.skip("library not built")
    st, site, index, unit, count = sr.sr_bounds_report()
    assert st == sr.SR_ERR_UNSUPPORTED and site == -1 and count == 0


def test_checked_kernel_file_compiles(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    csrc = os.path.join(ROOT, "paper_1807_07433_gb300", "csrc")
    r = subprocess.run([nvcc, "-c", os.path.join(csrc, "k_pixel.cu"), "-o", str(tmp_path / "k.o"),
                        "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                        "-I", csrc, "-gencode", "arch=compute_103a,code=sm_103a",
                        "-DSR_BOUNDS_CHECK"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
