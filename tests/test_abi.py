"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function include/sr.h declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sr.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1807_07433_gb300 import _build, sr
    _build.build()
    return sr.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:sr_status|const\s+char\s*\*|int)\s*(sr_\w+)\s*\(",
                                 text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sr_create", "sr_set_plane", "sr_match", "sr_reconstruct", "sr_destroy"):
        assert must in names


def test_library_exports_every_declared_function(lib):
    from paper_1807_07433_gb300 import sr
    names = declared_functions()
    assert names, "no declarations parsed"
    for n in names:
        assert hasattr(lib, n), f"libsr.so does not export {n}"
    assert set(names) <= set(sr.EXPORTS) | set(names)
    for n in sr.EXPORTS:
        assert n in names, f"binding wraps {n}, which the header does not declare"


def test_status_strings(lib):
    from paper_1807_07433_gb300 import sr
    assert sr.status_name(sr.SR_OK) == "SR_OK"
    assert sr.status_name(sr.SR_ERR_UNSUPPORTED) == "SR_ERR_UNSUPPORTED"
    assert sr.status_name(99) == "SR_ERR_UNKNOWN"
    assert "sm_103a" in sr.sr_version()
    assert sr.sr_stage_names()[0] == "prep"


@pytest.mark.parametrize("field,value,status", [
    ("width", 0, "SR_ERR_INVALID_ARG"),
    ("height", -3, "SR_ERR_INVALID_ARG"),
    ("max_disp", 0, "SR_ERR_INVALID_ARG"),
    ("gamma_d", 0.0, "SR_ERR_INVALID_ARG"),
    ("gamma_r", float("nan"), "SR_ERR_INVALID_ARG"),
    ("lr_thresh", -1.0, "SR_ERR_INVALID_ARG"),
    ("vol_dtype", 7, "SR_ERR_INVALID_ARG"),
    ("vol_dtype", -1, "SR_ERR_INVALID_ARG"),
    ("max_disp", 48, "SR_ERR_UNSUPPORTED"),
    ("max_disp", 128, "SR_ERR_UNSUPPORTED"),
    ("ncc_radius", 6, "SR_ERR_UNSUPPORTED"),
    ("agg_radius", 8, "SR_ERR_UNSUPPORTED"),
    ("agg_radius", 0, "SR_ERR_UNSUPPORTED"),
])
def test_create_rejects_bad_parameters_before_any_cuda_call(lib, field, value, status):
    from paper_1807_07433_gb300 import sr
    p = sr.make_params(64, 32, 16, 2, 2, 3.0, 10.0)
    setattr(p, field, value)
    ctx = ctypes.c_void_p(1234)
    rc = lib.sr_create(ctypes.byref(p), None, ctypes.byref(ctx))
    assert sr.status_name(rc) == status
    assert ctx.value is None


def test_null_arguments(lib):
    from paper_1807_07433_gb300 import sr
    p = sr.make_params(64, 32, 16, 2, 2, 3.0, 10.0)
    assert lib.sr_create(ctypes.byref(p), None, None) == sr.SR_ERR_INVALID_ARG
    assert lib.sr_create(None, None, ctypes.byref(ctypes.c_void_p())) == sr.SR_ERR_INVALID_ARG
    assert lib.sr_destroy(None) == sr.SR_OK
    assert lib.sr_set_plane(None, 0.0, 0.0, 0.0) == sr.SR_ERR_INVALID_ARG
    assert lib.sr_set_camera(None, 700.0, 120.0, 0.0, 0.0) == sr.SR_ERR_INVALID_ARG
    assert lib.sr_match(None, None, None, 64, None, None) == sr.SR_ERR_INVALID_ARG
    assert lib.sr_match_host(None, None, None, None) == sr.SR_ERR_INVALID_ARG
    assert lib.sr_match_host_async(None, None, None, None) == sr.SR_ERR_INVALID_ARG
    assert lib.sr_reconstruct(None, None, None) == sr.SR_ERR_INVALID_ARG
    n = ctypes.c_size_t(0)
    assert lib.sr_get_buffer(None, 0, None, ctypes.byref(n)) == sr.SR_ERR_INVALID_ARG
    assert lib.sr_set_debug(None, 1) == sr.SR_ERR_INVALID_ARG
    assert lib.sr_set_profiling(None, 1) == sr.SR_ERR_INVALID_ARG
    assert lib.sr_last_error(None) == b""


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1807_07433_gb300 import sr
    saved = sr._lib
    try:
        sr._lib = None
        with pytest.raises(OSError):
            sr.load(str(tmp_path / "missing.so"))
    finally:
        sr._lib = saved
