"""The R-SVD form (Sec. 2.2) through the C ABI.

Sigma V' of R is compared element by element with the oracle's one-sided
Jacobi (oracle.r_svd, itself pinned against LAPACK and a closed form), and
pinned by what the SVD fixes, not by an implementation:
  * sigma equals LAPACK's singular values of the same R (relative 1e-12 of sigma_max);
  * (Sigma V')' (Sigma V') = R' R (relative 1e-12): Sigma V' = U' R with U orthogonal;
  * the rows are orthogonal: (Sigma V')(Sigma V')' = Sigma^2 (off-diagonal 1e-12 of sigma_max^2);
  * Sec. 2.2: SPA and XRAY pick the same K on Sigma V' as on R.
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


@pytest.mark.parametrize("m,n", [(10, 1), (100, 7), (5000, 50), (3000, 101), (8000, 200), (2000, 256)])
def test_r_svd_invariants(h, oracle, m, n):
    X = synth.random_nonneg(m, n, seed=11 * n)
    Ro = oracle.qr_r(X.astype(np.float64))
    sig, SVt = h.r_svd(dev(Ro))
    h.sync()
    s, S = host(sig), host(SVt)
    sl = np.linalg.svd(Ro, compute_uv=False)
    assert np.all(np.diff(s) <= 0)
    np.testing.assert_allclose(s, sl, rtol=0, atol=1e-12 * sl[0])
    G = Ro.T @ Ro
    assert np.linalg.norm(S.T @ S - G) <= 1e-12 * np.linalg.norm(G)
    D = S @ S.T
    assert np.max(np.abs(D - np.diag(np.diag(D)))) <= 1e-12 * sl[0] ** 2
    np.testing.assert_allclose(np.sqrt(np.diag(D)), s, rtol=1e-12, atol=1e-12 * sl[0])


@pytest.mark.parametrize("m,n", [(100, 7), (5000, 50), (3000, 101), (8000, 200), (2000, 256)])
def test_r_svd_matches_oracle(h, oracle, m, n):
    """Element by element against the oracle's one-sided Jacobi (binary64,
    its own cyclic pair order): sigma within 1e-12 sigma_max, and every row of
    Sigma V' after aligning its sign, within 1e-12 sigma_max^2 / gap_i where
    gap_i is the distance from sigma_i to its nearest neighbour (first-order
    perturbation of a singular vector: error / sigma_max ~ eps sigma_max /
    gap).  Rows whose gap is below 1e-6 sigma_max, whose bound would say
    nothing, are left to the invariants above."""
    X = synth.random_nonneg(m, n, seed=13 * n + 1)
    Ro = oracle.qr_r(X.astype(np.float64))
    sig, SVt = h.r_svd(dev(Ro))
    h.sync()
    so, So, st = oracle.r_svd(Ro)
    assert st == 0
    s, S = host(sig), host(SVt)
    np.testing.assert_allclose(s, so, rtol=0, atol=1e-12 * so[0])
    checked = 0
    for i in range(n):
        gap = min([abs(so[i] - so[j]) for j in (i - 1, i + 1) if 0 <= j < n], default=so[0])
        if gap > 1e-6 * so[0]:
            sgn = 1.0 if S[i] @ So[i] >= 0 else -1.0
            np.testing.assert_allclose(sgn * S[i], So[i], rtol=0, atol=1e-12 * so[0] ** 2 / gap)
            checked += 1
    assert checked >= n // 2


def test_r_svd_rank_deficient(h, oracle):
    X, P = synth.planted_separable(20000, 30, 5, seed=1402001, dtype=np.float64)
    Ro = oracle.qr_r(X)
    sig, SVt = h.r_svd(dev(Ro))
    h.sync()
    s = host(sig)
    assert np.all(s[5:] <= 1e-10 * s[0])


@pytest.mark.parametrize("method", ["spa", "xray"])
def test_selection_on_svt_matches_r(h, oracle, method):
    # Sec. 2.2: K is invariant under the left orthogonal factor U'
    X, P = synth.planted_separable(60000, 48, 9, seed=21, noise=1e-3)
    X64 = X.astype(np.float64)
    Ro = oracle.qr_r(X64)
    cs = oracle.colsum(X64)
    sig, SVt = h.r_svd(dev(Ro))
    Kr, _ = h.select_extreme(method, R=dev(Ro), colsum=dev(cs), r=9)
    Ks, _ = h.select_extreme(method, R=SVt, colsum=dev(cs), r=9)
    h.sync()
    assert list(host(Kr)) == list(host(Ks))
    if method == "spa":
        assert sorted(host(Ks)) == list(P.K)
