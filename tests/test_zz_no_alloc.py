"""mrnmf_tsqr_r_noalloc against mrnmf_tsqr_r.

The no-alloc entry point serves callers that cannot call cudaMalloc (code in
host callbacks or allocator hooks, or under an application-owned memory pool):
its scratch is a fixed __device__ array in the library.  Its R and column sums
must match those of the ordinary, handle-based entry point within the FP32
pass tolerance used throughout the tests (relative Frobenius 1e-5 for R,
relative 1e-6 for the column sums), on two calls in a row -- the second with a
different shape, so stale contents of the shared array would show.

This file is collected last so that a run stopping at its first failure has
already run every other test; it passes alone in a fresh process too.
"""
import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R_TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_6964_gb300 import build, mrnmf
    build.build()
    return mrnmf


def test_noalloc_matches_handle_entry_point(lib):
    mrnmf = lib
    h = mrnmf.Handle()
    for m, n, seed in [(300_001, 50, 1), (70_003, 20, 2)]:
        X = torch.from_numpy(synth.random_nonneg(m, n, seed=seed)).cuda()
        R = torch.empty((n, n), dtype=torch.float64, device="cuda")
        cs = torch.empty(n, dtype=torch.float64, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        assert mrnmf.tsqr_r_noalloc(X, R, cs, status) == mrnmf.OK
        R_ref, cs_ref = h.tsqr_r(X, prec="fp32")
        h.sync()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        Rn, Rr = R.cpu().numpy(), R_ref.cpu().numpy()
        assert np.linalg.norm(Rn - Rr) / np.linalg.norm(Rr) <= R_TOL_FP32
        np.testing.assert_allclose(cs.cpu().numpy(), cs_ref.cpu().numpy(), rtol=1e-6)
    h.close()


def test_noalloc_rejects_bad_arguments(lib):
    mrnmf = lib
    X = torch.zeros((10, 300), dtype=torch.float32, device="cuda")
    R = torch.empty((300, 300), dtype=torch.float64, device="cuda")
    assert mrnmf.tsqr_r_noalloc(X, R) == mrnmf.ERR_INVALID_ARG  # n > 256 (and m < n)
