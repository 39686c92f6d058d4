"""Host-only checks of the C ABI: the library loads, exports what the header
declares, and rejects bad arguments before touching the GPU."""
import ctypes

import numpy as np
import pytest

from paper_2605_07954_gb300 import _capi


@pytest.fixture(scope="module")
def lib():
    from paper_2605_07954_gb300 import build
    build.build()
    return _capi.load()


def test_exports_every_declared_symbol(lib):
    names = _capi.declared_symbols()
    assert "stencil_run" in names and "stencil_plan_create" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def test_version_and_status_strings(lib):
    assert lib.stencil_version() >= 100
    for code in range(7):
        assert lib.stencil_status_string(code).decode().startswith("STENCIL_")


def _create(lib, ny, nx, r, w, dtype=0, boundary=0, opt=None):
    h = ctypes.c_void_p()
    wp = None if w is None else w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    st = lib.stencil_plan_create(ctypes.byref(h), ny, nx, r, wp, dtype, boundary,
                                 ctypes.byref(opt) if opt is not None else None)
    return st, h


@pytest.mark.parametrize("args,expect", [
    ((0, 8, 1), _capi.STENCIL_ERR_INVALID_ARG),
    ((8, 0, 1), _capi.STENCIL_ERR_INVALID_ARG),
    ((8, 8, 0), _capi.STENCIL_ERR_INVALID_ARG),
    ((8, 8, 4), _capi.STENCIL_ERR_UNSUPPORTED),
])
def test_rejects_bad_sizes(lib, args, expect):
    w = np.ones((9, 9), dtype=np.float32)
    st, h = _create(lib, *args, w)
    assert st == expect and not h.value
    assert lib.stencil_last_error().decode() != ""


def test_rejects_null_and_bad_enums(lib):
    w = np.ones((3, 3), dtype=np.float32)
    assert _create(lib, 8, 8, 1, None)[0] == _capi.STENCIL_ERR_INVALID_ARG
    assert _create(lib, 8, 8, 1, w, dtype=7)[0] == _capi.STENCIL_ERR_INVALID_ARG
    assert _create(lib, 8, 8, 1, w, boundary=5)[0] == _capi.STENCIL_ERR_INVALID_ARG
    bad = np.array([[0, 1, 0], [1, np.nan, 1], [0, 1, 0]], dtype=np.float32)
    assert _create(lib, 8, 8, 1, bad)[0] == _capi.STENCIL_ERR_INVALID_ARG
    opt = _capi.stencil_options_t(0, 9, 0, 0, 0, 0)
    assert _create(lib, 8, 8, 1, w, opt=opt)[0] == _capi.STENCIL_ERR_INVALID_ARG
    for field, value in (("compute", 6), ("kernel", 7), ("mma_n", -1), ("timeout_ms", -5),
                         ("debug_withhold", 2), ("load", 3), ("load", -1),
                         ("rank", -1), ("rank", 4)):
        opt = _capi.stencil_options_t()
        setattr(opt, field, value)
        assert _create(lib, 8, 8, 1, w, opt=opt)[0] == _capi.STENCIL_ERR_INVALID_ARG, field
    assert lib.stencil_plan_create(None, 8, 8, 1, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                   0, 0, None) == _capi.STENCIL_ERR_INVALID_ARG


def test_null_plan_calls(lib):
    assert lib.stencil_run(None, None, None, 1, None) == _capi.STENCIL_ERR_INVALID_ARG
    assert lib.stencil_run_host(None, None, None, 1, None) == _capi.STENCIL_ERR_INVALID_ARG
    assert lib.stencil_plan_status(None) == _capi.STENCIL_ERR_INVALID_ARG
    assert lib.stencil_run_launches(None, 3) == -1
    lib.stencil_plan_destroy(None)
