"""The optional second-read follow-ups (gather W = X(:,K), full-space residual)
through the C ABI, against numpy indexing and the FP64 oracle.

  gather        : bit-exact
  full residual : F64 X: relative 1e-10 against the oracle's residual of X;
                  F32 X: relative 1e-3 (binary32 residual of a near-separable
                  fit, where E = X - X(:,K)H is ~1e-3 of X: cancellation costs
                  about three of binary32's seven digits)
  Sec. 2.4      : the full-space residual equals the reduced one on R
"""
import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_6964_gb300 import build, mrnmf
    build.build()
    hd = mrnmf.Handle()
    yield hd
    hd.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("m,n", [(1, 1), (777, 13), (100003, 50), (4099, 256)])
def test_gather_columns_exact(h, m, n, dtype):
    X = synth.random_nonneg(m, n, seed=m + n).astype(dtype)
    rng = np.random.default_rng(n)
    K = rng.choice(n, size=min(n, 7), replace=False).astype(np.int32)
    W = h.gather_columns(dev(X), dev(K))
    h.sync()
    assert np.array_equal(host(W), X[:, K])


def test_gather_columns_strided(h):
    Wd = dev(synth.random_nonneg(3000, 40, seed=5))
    Xd = Wd[:, 3:33]
    K = np.array([29, 0, 7], np.int32)
    W = h.gather_columns(Xd, dev(K))
    h.sync()
    assert np.array_equal(host(W), host(Xd)[:, K])


@pytest.fixture(scope="module")
def fit(oracle):
    X, P = synth.planted_separable(60000, 48, 9, seed=21, noise=1e-3)
    X64 = X.astype(np.float64)
    Ro = oracle.qr_r(X64)
    Ko, _ = oracle.spa(Ro, oracle.colsum(X64), 9)
    Ho, _ = oracle.nnls_h(Ro, Ko)
    return X, X64, Ro, Ko, Ho


def test_full_residual_f64_matches_oracle(h, oracle, fit):
    X, X64, Ro, Ko, Ho = fit
    out = h.full_residual(dev(X64), dev(Ko), dev(Ho))
    h.sync()
    ab, rel = oracle.residual(X64, Ko, Ho)
    assert host(out)[0] == pytest.approx(ab, rel=1e-10)
    assert host(out)[1] == pytest.approx(rel, rel=1e-10)
    # Sec. 2.4: the same as the reduced residual on R
    ab_r, rel_r = oracle.residual(Ro, Ko, Ho)
    assert host(out)[0] == pytest.approx(ab_r, rel=1e-8)


def test_full_residual_f32_matches_oracle(h, oracle, fit):
    X, X64, Ro, Ko, Ho = fit
    out = h.full_residual(dev(X), dev(Ko), dev(Ho))
    h.sync()
    ab, rel = oracle.residual(X64, Ko, Ho)
    assert host(out)[0] == pytest.approx(ab, rel=1e-3)
    assert host(out)[1] == pytest.approx(rel, rel=2e-3)


@pytest.mark.parametrize("n", [20, 100, 256])
def test_full_residual_exact_separable_is_zero(h, oracle, n):
    # noise-free separable X (Sec. 4): X = X(:,K) H exactly, so the residual is rounding
    X, P = synth.planted_separable(20000, n, 5, seed=1402001 + n, dtype=np.float64)
    out = h.full_residual(dev(X), dev(P.K), dev(P.H_true))
    h.sync()
    assert host(out)[1] <= 1e-24


def test_full_residual_bad_index_is_reported(h):
    from paper_1402_6964_gb300 import mrnmf
    X = synth.random_nonneg(1000, 10, seed=3)
    K = np.array([2, 11], np.int32)
    H = np.zeros((2, 10))
    h.full_residual(dev(X), dev(K), dev(H))
    with pytest.raises(mrnmf.MrnmfError) as e:
        h.sync()
    assert e.value.status == mrnmf.ERR_INVALID_ARG


def test_kron_stream_matches_oracle(h, oracle):
    # X = A kron A (the structure of Sec. 5.2's flow-cytometry matrix), streamed in chunks
    w = synth.WORKLOADS["kron_fc_1p6e9x25"]
    A, Kp = synth.kron_factor(w, rows=600)
    At = torch.from_numpy(A.astype(np.float32)).cuda()
    m = 600 * 600
    h.stream_begin(25, k=w.k, seed=w.seed)
    for a in range(0, m, 100_000):
        h.stream_push(synth.kron_rows(At, a, min(100_000, m - a)))
    R, cs, GX = h.stream_end(25, k=w.k)
    K, gap = h.select_extreme("spa", R=R, colsum=cs, r=16)
    h.sync()
    # the oracle gets the same binary32 rows the pass read (A kron A is near
    # rank-deficient, cond ~1e6, so rounding the products differently moves
    # R's small rows); R is checked through the Gram identity R'R = X'X
    X64 = synth.kron_rows(torch.from_numpy(A.astype(np.float32)), 0, m).numpy().astype(np.float64)
    Ro = oracle.qr_r(X64)
    Rg = host(R)
    G = X64.T @ X64
    assert np.linalg.norm(Rg.T @ Rg - G) <= 2e-5 * np.linalg.norm(G)
    assert np.linalg.norm(Rg.T @ Rg - Ro.T @ Ro) <= 2e-5 * np.linalg.norm(G)
    np.testing.assert_allclose(host(cs), oracle.colsum(X64), rtol=1e-6)
    Ko, go = oracle.spa(Ro, oracle.colsum(X64), 16)
    assert sorted(host(K).tolist()) == sorted(Ko.tolist())
    assert sorted(Ko.tolist()) == Kp.tolist()
