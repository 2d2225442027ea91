"""Host-side checks of the user-function entry points: argument validation,
and NVRTC compilation of the test functions for sm_103a (which needs no GPU:
without one, a source that compiles fails only at loading, with
CHESSFAD_ERR_CUDA, while a source that does not compile fails with
CHESSFAD_ERR_JIT and NVRTC's message)."""
import ctypes

import pytest

import paper_2410_22575_gb300 as cf

from user_sources import SOURCES


def _gpu():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def test_argument_errors():
    lib = cf.load()
    h = ctypes.c_void_p()
    src, name = SOURCES[0]
    assert lib.chessfad_user_fn_create(None, b"f", 4, 0, ctypes.byref(h), None, 0) == -5
    assert lib.chessfad_user_fn_create(src.encode(), None, 4, 0, ctypes.byref(h), None, 0) == -5
    assert lib.chessfad_user_fn_create(src.encode(), name.encode(), 4, 0, None, None, 0) == -5
    assert lib.chessfad_user_fn_create(src.encode(), name.encode(), 3, 0, ctypes.byref(h), None, 0) == -4
    assert lib.chessfad_user_fn_create(src.encode(), name.encode(), 64, 0, ctypes.byref(h), None, 0) == -4
    assert lib.chessfad_user_fn_create(src.encode(), name.encode(), 4, 5, ctypes.byref(h), None, 0) == -7
    st, handle, log = cf.chessfad_user_fn_create(src, "not an identifier", 4, 0)
    assert st == -12 and handle is None and "identifier" in log
    d = ctypes.c_void_p(16)
    assert lib.chessfad_user_hvp(None, 8, 4, d, d, d, None, None) == -5
    assert lib.chessfad_user_hessian(None, 8, 4, d, d, None, None) == -5
    assert lib.chessfad_user_fn_destroy(None) == 0
    assert cf.strerror(-12) != "unknown status"


def test_compile_error_is_reported():
    st, handle, log = cf.chessfad_user_fn_create(
        "template <class R, class X> R bad(const X &x, int n, const double *p) { return x[0] + undefined_name; }",
        "bad", 4, cf.FP64)
    assert st == -12 and handle is None
    assert "undefined_name" in log and "user_function" in log


@pytest.mark.parametrize("fn", sorted(SOURCES))
@pytest.mark.parametrize("prec", [cf.FP64, cf.FP32_COMP])
def test_test_functions_compile(fn, prec):
    src, name = SOURCES[fn]
    st, handle, log = cf.chessfad_user_fn_create(src, name, 8, prec)
    if _gpu():
        assert st == 0, log
        cf.chessfad_user_fn_destroy(handle)
    else:
        assert st == -10, (st, log)  # compiled; no device to load it on
        assert log.startswith("compiled")
