"""The Python binding's own checks (no GPU): it rejects host tensors where the
C ABI takes device memory, non-row-major layouts, unsupported dtypes and
device memory where it takes host memory, before calling the library, and
argument errors the library reports surface as MrnmfError with their status."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


class _NoStream:
    """Stands in for a torch stream on a machine without CUDA (the legacy
    default stream, which the library never touches on an argument error)."""
    cuda_stream = 0


@pytest.fixture(scope="module")
def mrnmf():
    from paper_1402_6964_gb300 import build, mrnmf as m
    build.build()
    return m


def test_host_tensors_are_refused(mrnmf):
    with mrnmf.Handle() as h:
        X = torch.rand(100, 8)
        for call in (lambda: h.tsqr_r(X), lambda: h.gauss_project(X, 4, 1), lambda: h.tsqr_gp(X, 4, 1),
                     lambda: h.stream_push(X)):
            with pytest.raises(ValueError):
                call()


def test_layout_and_dtype_checks(mrnmf):
    from paper_1402_6964_gb300.mrnmf import _check_X, _dtype_code
    with pytest.raises(ValueError):
        _check_X(torch.rand(8))
    with pytest.raises(TypeError):
        _dtype_code(torch.zeros(4, 4, dtype=torch.int32))
    assert _dtype_code(torch.zeros(2, 2, dtype=torch.float64)) == mrnmf.F64


def test_library_argument_errors_raise_with_status(mrnmf):
    with mrnmf.Handle() as h:
        with pytest.raises(mrnmf.MrnmfError) as e:
            h.stream_end(8, device="cpu", stream=_NoStream())  # no open stream
        assert e.value.status == mrnmf.ERR_INVALID_ARG
        with pytest.raises(mrnmf.MrnmfError) as e:
            h.stream_state_save()
        assert e.value.status == mrnmf.ERR_INVALID_ARG
        assert "stream" in str(e.value)


def test_selftest_wrappers_reject_bad_arguments(mrnmf):
    with pytest.raises(mrnmf.MrnmfError):
        mrnmf.wait_selftest(7, 5_000_000, device="cpu", stream=_NoStream())
