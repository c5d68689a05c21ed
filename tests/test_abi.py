"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every symbol include/mrnmf.h declares, and rejects
bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1402_6964_gb300 import build, mrnmf
    build.build()
    return mrnmf.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "mrnmf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrnmf_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ["mrnmf_tsqr_r", "mrnmf_gauss_project", "mrnmf_select_extreme", "mrnmf_nnls_h", "mrnmf_residual"]:
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1402_6964_gb300 import mrnmf
    names = _declared()
    missing = [s for s in names if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(mrnmf.EXPORTS) == sorted(s for s in names if s in mrnmf.EXPORTS)


def test_argument_errors_need_no_device(lib):
    from paper_1402_6964_gb300 import mrnmf
    h = ctypes.c_void_p()
    assert lib.mrnmf_create(ctypes.byref(h)) == 0
    dummy = ctypes.c_void_p(16)
    # m < n, n out of range, ldx < n, NULL X, bad dtype / prec / k
    assert lib.mrnmf_tsqr_r(h, dummy, 4, 5, 5, 0, 0, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_tsqr_r(h, dummy, 1000, 0, 5, 0, 0, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_tsqr_r(h, dummy, 1000, 257, 300, 0, 0, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_tsqr_r(h, dummy, 1000, 8, 7, 0, 0, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_tsqr_r(h, None, 1000, 8, 8, 0, 0, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_tsqr_r(h, dummy, 1000, 8, 8, 5, 0, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_tsqr_r(h, dummy, 1000, 8, 8, 0, 9, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_gauss_project(h, dummy, 1000, 8, 8, 0, 0, 1, 0, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_gauss_project(h, dummy, 1000, 8, 8, 0, 65, 1, 0, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    # tensor-core projection: a form other than TF32X3 / BF16, n > 128, k = 0, no GX
    for form in (0, 1, 2, 5):
        assert lib.mrnmf_gauss_project_tc(h, dummy, 1000, 8, 8, 4, 1, 0, form, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_gauss_project_tc(h, dummy, 1000, 129, 129, 4, 1, 0, 4, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_gauss_project_tc(h, dummy, 1000, 8, 8, 0, 1, 0, 4, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_gauss_project_tc(h, dummy, 1000, 8, 8, 4, 1, 0, 4, None, None, None) == mrnmf.ERR_INVALID_ARG
    # BF16 is a form of the projection alone: the passes that form R reject it
    assert lib.mrnmf_tsqr_r(h, dummy, 1000, 8, 8, 0, 4, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    # selection: r > n, unknown method, GP without GX
    assert lib.mrnmf_select_extreme(h, 0, dummy, 8, dummy, None, 0, 9, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_select_extreme(h, 7, dummy, 8, dummy, None, 0, 3, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_select_extreme(h, 2, None, 8, dummy, None, 4, 3, dummy, None, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_nnls_h(h, dummy, 8, dummy, 0, dummy, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_residual(h, dummy, 8, dummy, 9, dummy, dummy, None) == mrnmf.ERR_INVALID_ARG
    # streaming misuse
    assert lib.mrnmf_stream_push(h, dummy, 10, 8, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_stream_end(h, dummy, None, None, None) == mrnmf.ERR_INVALID_ARG
    sz = ctypes.c_size_t(0)
    assert lib.mrnmf_stream_state_size(h, ctypes.byref(sz)) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_stream_state_save(h, dummy, 1 << 20, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_stream_state_load(h, dummy, 1 << 20, None) == mrnmf.ERR_INVALID_ARG
    # failure injection: a link outside 0..3, a limit outside [1e3, 1e9], NULL outputs
    assert lib.mrnmf_wait_selftest(4, 5000000, dummy, dummy, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_wait_selftest(1, 10, dummy, dummy, None) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_wait_selftest(1, 5000000, None, dummy, None) == mrnmf.ERR_INVALID_ARG
    msg = lib.mrnmf_last_error_string(h)
    assert isinstance(msg, bytes) and len(msg) > 0
    lib.mrnmf_destroy(h)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1402_6964_gb300 import mrnmf
    with pytest.raises(ImportError):
        mrnmf.load(str(tmp_path / "nope.so"))
