"""mrnmf_tsqr_r_noalloc against the FP64 oracle and the handle-based pass.

The no-alloc entry point serves callers that cannot call cudaMalloc: code that
runs inside a host callback or an allocator hook, or under a memory pool that
the embedding application owns outright.  Its scratch is a fixed __device__
array inside the library.  These tests check, on two or more calls in a row
with different shapes (so stale contents of the shared array would show):

* R against the oracle's FP64 Householder R within the FP32 pass tolerance
  (relative Frobenius 1e-5) and the column sums within relative 1e-6;
* R and the column sums against the ordinary entry point mrnmf_tsqr_r;
* shapes that reach each leaf: the lane-group leaf (n = 12), the warp leaf
  (n = 20, 50), the pipelined leaf (n = 100), and n = 256, where the state of the usual stream count does not
  fit the array, so the call runs fewer streams and the fan-in-2 tree;
* that a call allocates no device memory (torch's allocator and the driver's
  free-memory count do not grow across it);
* that a NULL status word is rejected.

This file is collected last so that a run stopping at its first failure has
already run every other test; it passes alone in a fresh process too.
"""
import gc

import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R_TOL_FP32 = 1e-5     # relative Frobenius error of R, FP32 pass
CS_RTOL = 1e-6        # column sums (binary64 partial sums of binary32 tile sums)

# (m, n, seed, decades): decades > 0 scales the columns by 10^U(0, decades)
CASES = [(300_001, 50, 1, 0.0), (70_003, 20, 2, 0.0), (200_000, 100, 3, 3.0), (40_000, 256, 4, 3.0),
         (150_007, 12, 5, 0.0)]


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_6964_gb300 import build, mrnmf
    build.build()
    return mrnmf


def _input(m, n, seed, decades):
    if decades > 0:
        X, _ = synth.planted_separable(m, n, max(2, n // 10), seed=1403000 + seed, noise=1e-3, decades=decades)
        return X
    return synth.random_nonneg(m, n, seed=seed)


def _noalloc(mrnmf, Xd, n):
    R = torch.empty((n, n), dtype=torch.float64, device="cuda")
    cs = torch.empty(n, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rc = mrnmf.tsqr_r_noalloc(Xd, R, cs, status)
    return rc, R, cs, status


def test_noalloc_matches_oracle_and_handle_entry_point(lib, oracle):
    mrnmf = lib
    h = mrnmf.Handle()
    for m, n, seed, decades in CASES:
        X = _input(m, n, seed, decades)
        Xd = torch.from_numpy(X).cuda()
        rc, R, cs, status = _noalloc(mrnmf, Xd, n)
        assert rc == mrnmf.OK
        R_ref, cs_ref = h.tsqr_r(Xd, prec="fp32")
        h.sync()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        Rn, csn = R.cpu().numpy(), cs.cpu().numpy()
        X64 = X.astype(np.float64)
        Ro = oracle.qr_r(X64)
        err = np.linalg.norm(Rn - Ro) / np.linalg.norm(Ro)
        assert err <= R_TOL_FP32, (m, n, err)
        np.testing.assert_allclose(csn, oracle.colsum(X64), rtol=CS_RTOL)
        Rr = R_ref.cpu().numpy()
        assert np.linalg.norm(Rn - Rr) / np.linalg.norm(Rr) <= R_TOL_FP32
        np.testing.assert_allclose(csn, cs_ref.cpu().numpy(), rtol=CS_RTOL)
    h.close()


def test_noalloc_allocates_nothing(lib):
    mrnmf = lib
    for m, n, seed, decades in [(300_001, 50, 5, 0.0), (40_000, 256, 6, 0.0)]:
        Xd = torch.from_numpy(_input(m, n, seed, decades)).cuda()
        R = torch.empty((n, n), dtype=torch.float64, device="cuda")
        cs = torch.empty(n, dtype=torch.float64, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        # a first call loads the kernels this shape uses (lazy module loading)
        assert mrnmf.tsqr_r_noalloc(Xd, R, cs, status) == mrnmf.OK
        torch.cuda.synchronize()
        R0 = R.clone()
        gc.collect()
        torch.cuda.synchronize()
        used0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
        assert mrnmf.tsqr_r_noalloc(Xd, R, cs, status) == mrnmf.OK
        torch.cuda.synchronize()
        # neither torch's allocator nor the driver gave out memory during the call
        assert torch.cuda.memory_allocated() <= used0
        assert torch.cuda.mem_get_info()[0] >= free0
        assert int(status.item()) == 0
        assert torch.equal(R, R0)  # same input, same result: no state leaks between calls


def test_noalloc_rejects_bad_arguments(lib):
    mrnmf = lib
    X = torch.zeros((10, 300), dtype=torch.float32, device="cuda")
    R = torch.empty((300, 300), dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert mrnmf.tsqr_r_noalloc(X, R, status=status) == mrnmf.ERR_INVALID_ARG  # n > 256 (and m < n)
    X = torch.ones((100, 8), dtype=torch.float32, device="cuda")
    R = torch.empty((8, 8), dtype=torch.float64, device="cuda")
    assert mrnmf.tsqr_r_noalloc(X, R) == mrnmf.ERR_INVALID_ARG  # no status word
