"""Pins for the FP64 oracle, checked against facts fixed outside it.

Each test names the passage of the paper (arXiv 1402.6964) or the textbook
fact it relies on.  None of them compares the oracle with itself: the
expected values come from hand-worked fixtures in tests/golden, exact integer
arithmetic, closed forms, library routines of a different algorithm, or brute
force.
"""
import itertools
import math
import os

import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = {}
    cases = [{}]
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line == "---":
            cases.append({})
            continue
        tag, *vals = line.split()
        cases[-1].setdefault(tag, []).append([float(v) for v in vals])
    return cases


# ---------------------------------------------------------------- R (Sec. 3.1)

def test_qr_hand_cases(oracle):
    for case in _read("qr_hand.txt"):
        X = np.array(case["X"])
        R = oracle.qr_r(X)
        np.testing.assert_allclose(R, np.array(case["R"]), rtol=0, atol=1e-14)


def test_qr_gram_exact_integer(oracle):
    # R^T R = X^T X; for small-integer X the Gram is exact in int64.
    X = synth.random_nonneg(300, 9, seed=11, dtype=np.float64, integer=True)
    R = oracle.qr_r(X)
    G = X.astype(np.int64).T @ X.astype(np.int64)
    np.testing.assert_allclose(R.T @ R, G.astype(np.float64), rtol=1e-13, atol=1e-10)
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.all(np.diag(R) >= 0.0)


def test_qr_equals_cholesky_of_gram(oracle):
    # For full-rank, well-conditioned X the unique R with positive diagonal is
    # chol(X^T X)^T -- a different algorithm (numpy/LAPACK Cholesky).
    X = synth.random_nonneg(500, 12, seed=12, dtype=np.float64)
    R = oracle.qr_r(X)
    L = np.linalg.cholesky(X.T @ X)
    np.testing.assert_allclose(R, L.T, rtol=1e-10, atol=1e-10)


def test_qr_orthogonal_invariance(oracle):
    # R(QX) = R(X) for orthogonal Q (Sec. 2.2: the reduction only sees Q^T X).
    X = synth.random_nonneg(60, 7, seed=13, dtype=np.float64)
    Q, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((60, 60)))
    np.testing.assert_allclose(oracle.qr_r(Q @ X), oracle.qr_r(X), rtol=1e-11, atol=1e-11)


def test_qr_tree_property(oracle):
    # TSQR's reduction (Sec. 3.1): R([X1; X2]) = R([R(X1); R(X2)]).
    X = synth.random_nonneg(400, 10, seed=14, dtype=np.float64)
    R = oracle.qr_r(X)
    R1 = oracle.qr_r(X[:170])
    R2 = oracle.qr_r(X[170:])
    np.testing.assert_allclose(oracle.qr_r(np.vstack([R1, R2])), R, rtol=1e-11, atol=1e-11)


def test_qr_rank_deficient_gram(oracle):
    # Exactly separable X has rank r < n; R^T R = X^T X still holds and rows
    # r..n-1 of R vanish to rounding.
    X, P = synth.planted_separable(2000, 12, 4, seed=15, dtype=np.float64)
    R = oracle.qr_r(X)
    np.testing.assert_allclose(R.T @ R, X.T @ X, rtol=1e-12, atol=1e-9)
    assert np.linalg.norm(R[4:]) < 1e-10 * np.linalg.norm(R)


def test_qr_transposed_operand_is_caught(oracle):
    # A planted mistake (returning R^T) must fail the Gram pin above.
    X = synth.random_nonneg(50, 5, seed=16, dtype=np.float64)
    R = oracle.qr_r(X)
    assert not np.allclose(R @ R.T, X.T @ X, rtol=1e-6)


# ---------------------------------------------------------- colsum (Sec. 3.3)

def test_colsum_exact(oracle):
    X = synth.random_nonneg(1000, 6, seed=17, dtype=np.float64, integer=True)
    np.testing.assert_array_equal(oracle.colsum(X), X.astype(np.int64).sum(0).astype(np.float64))
    # Kahan against an exactly rounded sum (math.fsum) on badly scaled data
    Y = np.abs(np.random.default_rng(3).standard_normal((20000, 3))) * 10.0 ** np.random.default_rng(4).uniform(-8, 8, (20000, 3))
    s = oracle.colsum(Y)
    for j in range(3):
        assert s[j] == pytest.approx(math.fsum(Y[:, j]), rel=1e-15)


# ------------------------------------------------------- Gaussian projection

def test_philox_known_answers(oracle):
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_gaussian_distribution(oracle):
    # g_i ~ N(0, I_k) (Algorithm 1): moments, a KS test, and no correlation
    # between the k coordinates of one row or between neighbouring rows.
    from scipy import stats
    G = oracle.gauss_matrix(seed=99, row0=0, rows=50000, k=8)
    z = G.ravel()
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-3
    C = np.corrcoef(G.T)
    assert np.max(np.abs(C - np.eye(8))) < 0.03
    assert abs(np.corrcoef(G[:-1, 0], G[1:, 0])[0, 1]) < 0.03
    # depends only on (seed, global row, coordinate): a later block is a slice
    np.testing.assert_array_equal(oracle.gauss_matrix(99, 1234, 10, 8), G[1234:1244])


def test_gauss_project_matches_matmul(oracle):
    # GX = G^T X: the row-by-row reduce of Algorithm 1 equals one matrix product
    X = synth.random_nonneg(700, 9, seed=18, dtype=np.float64)
    G = oracle.gauss_matrix(7, 100, 700, 6)
    np.testing.assert_allclose(oracle.gauss_project(X, 6, 7, row0=100), G.T @ X, rtol=1e-12, atol=1e-12)
    # commutation with the column scaling (Sec. 3.3): G^T (X D^-1) = (G^T X) D^-1
    d = np.arange(1, 10, dtype=np.float64)
    np.testing.assert_allclose(oracle.gauss_project(X / d, 6, 7, row0=100),
                               oracle.gauss_project(X, 6, 7, row0=100) / d, rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------- SPA (Sec. 2.1)

def test_spa_hand(oracle):
    c = _read("spa_hand.txt")[0]
    X = np.array(c["X"])
    K, gap = oracle.spa(X, X.sum(0), 2)
    assert list(K) == [int(v) for v in c["K"][0]]
    np.testing.assert_allclose(gap, c["GAP"][0], rtol=1e-12)


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_spa_recovers_planted(oracle, seed):
    # noise-free separable X: SPA recovers the planted extreme columns (Sec. 4)
    X, P = synth.planted_separable(3000, 20, 5, seed=seed, dtype=np.float64)
    R = oracle.qr_r(X)
    K, gap = oracle.spa(R, oracle.colsum(X), 5)
    assert sorted(K) == list(P.K)
    assert np.all(gap > 0)


def test_spa_on_R_equals_spa_on_X(oracle):
    # Sec. 2.2: SPA only uses column 2-norms, which Q^T preserves, so the
    # picks on R equal the picks on X itself.
    X, P = synth.planted_separable(1500, 16, 6, seed=24, noise=1e-3, dtype=np.float64)
    s = oracle.colsum(X)
    KX, _ = oracle.spa(X, s, 6)
    KR, _ = oracle.spa(oracle.qr_r(X), s, 6)
    assert list(KX) == list(KR)


def test_spa_column_scaling_invariance(oracle):
    # the l1 normalisation (Sec. 2.1) cancels any positive column scaling
    X, P = synth.planted_separable(800, 14, 4, seed=25, noise=1e-3, dtype=np.float64)
    d = 10.0 ** np.random.default_rng(1).uniform(-3, 3, 14)
    K1, _ = oracle.spa(X, X.sum(0), 4)
    K2, _ = oracle.spa(X * d, (X * d).sum(0), 4)
    assert list(K1) == list(K2)


def test_spa_bruteforce_unique_subset(oracle):
    # brute force over all r-subsets: exactly one has zero NNLS residual on an
    # exactly separable X, and it is what SPA returns (scipy's NNLS, a
    # different solver, decides the residual).
    from scipy.optimize import nnls as sp_nnls
    n, r = 10, 3
    X, P = synth.planted_separable(200, n, r, seed=26, dtype=np.float64)
    zero = []
    for S in itertools.combinations(range(n), r):
        A = X[:, S]
        res = sum(sp_nnls(A, X[:, j])[1] ** 2 for j in range(n))
        if res < 1e-16 * np.sum(X * X):
            zero.append(S)
    assert zero == [tuple(P.K)]
    K, _ = oracle.spa(oracle.qr_r(X), X.sum(0), r)
    assert tuple(sorted(K)) == zero[0]


# ------------------------------------------------------------ XRAY (Sec. 2.1)

def test_xray_hand(oracle):
    c = _read("xray_hand.txt")[0]
    X = np.array(c["X"])
    K, gap, st = oracle.xray(X, 2)
    assert st == 0
    assert list(K) == [int(v) for v in c["K"][0]]
    s = c["SCORE1"][0]
    assert gap[0] == pytest.approx((s[0] - s[2]) / s[0], rel=1e-12)
    H, st = oracle.nnls_h(X, K)
    np.testing.assert_allclose(H, np.array(c["H"]), atol=1e-14)


def test_xray_first_pick_closed_form(oracle):
    # step 1 with Res = X: argmax_j ||X^T x_j|| / ||x_j||, computed on X directly
    X, P = synth.planted_separable(900, 15, 5, seed=27, noise=1e-3, dtype=np.float64)
    G = X.T @ X
    scores = np.linalg.norm(G, axis=0) / np.sqrt(np.diag(G))
    K, gap, st = oracle.xray(oracle.qr_r(X), 3)
    assert K[0] == int(np.argmax(scores))


def test_xray_on_R_equals_xray_on_X(oracle):
    X, P = synth.planted_separable(1200, 14, 5, seed=28, noise=1e-3, dtype=np.float64)
    KX, _, _ = oracle.xray(X, 5)
    KR, _, _ = oracle.xray(oracle.qr_r(X), 5)
    assert list(KX) == list(KR)


@pytest.mark.parametrize("seed", range(3))
def test_xray_every_pick_is_the_scores_argmax(oracle, seed):
    # Sec. 2.1: after each pick, Res = X - X(:,K)H with H the NNLS fit of every
    # column (scipy's active-set NNLS here, a separate solver), and the next
    # pick maximises ||Res^T x_j|| / ||x_j|| over the unchosen columns
    from scipy.optimize import nnls as sp_nnls
    X, P = synth.planted_separable(400, 12, 5, seed=40 + seed, noise=1e-2, dtype=np.float64)
    r = 5
    K, gap, st = oracle.xray(X, r)
    assert st == 0
    chosen = []
    Res = X.copy()
    for t in range(r):
        scores = np.linalg.norm(Res.T @ X, axis=0) / np.linalg.norm(X, axis=0)
        scores[chosen] = -np.inf
        order = np.argsort(-scores, kind="stable")
        best, second = scores[order[0]], scores[order[1]]
        if (best - second) / best > 1e-9:  # clear pick: the rule fixes it
            assert K[t] == order[0], (t, K, order[:3])
        chosen.append(int(K[t]))
        A = X[:, chosen]
        H = np.stack([sp_nnls(A, X[:, c])[0] for c in range(X.shape[1])], axis=1)
        Res = X - A @ H


@pytest.mark.parametrize("seed", range(4))
def test_nnls_matches_scipy_for_larger_r(oracle, seed):
    # beyond brute-force sizes: the minimiser is unique (full column rank), so
    # it equals scipy's active-set NNLS solution
    from scipy.optimize import nnls as sp_nnls
    g = np.random.default_rng(200 + seed)
    m, r = 60, 24
    A = g.standard_normal((m, r))
    b = g.standard_normal(m)
    x, st = oracle.nnls(A.T @ A, A.T @ b, b @ b)
    assert st == 0
    np.testing.assert_allclose(x, sp_nnls(A, b)[0], rtol=1e-8, atol=1e-10)


# -------------------------------------------------------------- GP (Sec. 2.3)

def test_gp_hand(oracle):
    c = _read("gp_hand.txt")[0]
    GX = np.array(c["GX"])
    s = np.array(c["S"][0])
    K, cand, gap = oracle.gp_select(GX, s, 4)
    assert list(cand) == [int(v) for v in c["CAND"][0]]
    assert list(K) == [int(v) for v in c["CAND"][0]][:4]


def test_gp_candidates_are_extreme(oracle):
    # on noise-free separable data a linear functional over the simplex hull
    # of the l1-normalised columns peaks at a vertex: every candidate is a
    # planted extreme column (Sec. 2.3)
    X, P = synth.planted_separable(4000, 30, 6, seed=29, dtype=np.float64)
    GX = oracle.gauss_project(X, 12, seed=5)
    K, cand, gap = oracle.gp_select(GX, oracle.colsum(X), 6)
    assert set(cand) <= set(P.K)
    assert len(cand) >= 4


# ------------------------------------------------------------ NNLS (Sec. 2.4)

def _brute_nnls(A, b):
    # exact minimiser over all supports (unconstrained LS on each support,
    # keep the feasible one with the smallest residual)
    r = A.shape[1]
    best, bx = np.inf, None
    for mask in range(1 << r):
        S = [i for i in range(r) if mask >> i & 1]
        x = np.zeros(r)
        if S:
            xs, *_ = np.linalg.lstsq(A[:, S], b, rcond=None)
            if np.any(xs < 0):
                continue
            x[S] = xs
        res = np.sum((A @ x - b) ** 2)
        if bx is None or res < best - 1e-15 * max(1.0, best):
            best, bx = res, x
    return bx


@pytest.mark.parametrize("seed", range(6))
def test_nnls_bruteforce(oracle, seed):
    g = np.random.default_rng(100 + seed)
    m, r = 15, 7
    A = g.standard_normal((m, r))
    b = g.standard_normal(m)
    x, st = oracle.nnls(A.T @ A, A.T @ b, b @ b)
    assert st == 0
    np.testing.assert_allclose(x, _brute_nnls(A, b), rtol=1e-9, atol=1e-11)
    # KKT certificate
    w = A.T @ (b - A @ x)
    assert np.all(x >= 0)
    assert np.all(w <= 1e-9)
    assert np.all(np.abs(w[x > 0]) <= 1e-9)


def test_nnls_h_recovers_planted_H(oracle):
    # Sec. 2.4 / Sec. 4: on exact separable data H = the planted coefficients,
    # and the reduced NNLS equals the NNLS on X itself.
    X, P = synth.planted_separable(3000, 18, 5, seed=31, dtype=np.float64)
    R = oracle.qr_r(X)
    H, st = oracle.nnls_h(R, P.K)
    assert st == 0
    np.testing.assert_allclose(H, P.H_true, atol=1e-10)
    HX, st = oracle.nnls_h(X, P.K)
    np.testing.assert_allclose(H, HX, atol=1e-10)


def test_residual_reduced_equals_full(oracle):
    # Sec. 2.4: ||X - X(:,K)H|| = ||R - R(:,K)H||; 0 on exact data (Sec. 4)
    X, P = synth.planted_separable(2500, 16, 5, seed=32, noise=1e-2, dtype=np.float64)
    R = oracle.qr_r(X)
    K = P.K
    H, _ = oracle.nnls_h(R, K)
    full = np.linalg.norm(X - X[:, K] @ H)
    ab, rel = oracle.residual(R, K, H)
    assert ab == pytest.approx(full, rel=1e-9)
    assert rel == pytest.approx(full ** 2 / np.linalg.norm(X) ** 2, rel=1e-9)
    X0, P0 = synth.planted_separable(2500, 16, 5, seed=32, dtype=np.float64)
    R0 = oracle.qr_r(X0)
    H0, _ = oracle.nnls_h(R0, P0.K)
    assert oracle.residual(R0, P0.K, H0)[1] < 1e-20


# ------------------------------------------------------------------ R-SVD

def test_r_svd_golden_ratio(oracle):
    # closed form: R = [[1, 1], [0, 1]] has R'R = [[1, 1], [1, 2]], singular
    # values phi = (1 + sqrt 5)/2 and 1/phi, right singular vectors
    # [1, phi]/sqrt(1 + phi^2) and [-phi, 1]/sqrt(1 + phi^2)
    phi = (1 + 5 ** 0.5) / 2
    sig, S, st = oracle.r_svd(np.array([[1.0, 1.0], [0.0, 1.0]]))
    assert st == 0
    np.testing.assert_allclose(sig, [phi, 1 / phi], rtol=1e-15)
    d = (1 + phi ** 2) ** 0.5
    want = np.array([[phi * 1 / d, phi * phi / d], [-1 / phi * phi / d, 1 / phi * 1 / d]])
    for i in range(2):
        s = np.sign(S[i] @ want[i])
        np.testing.assert_allclose(s * S[i], want[i], rtol=1e-14, atol=1e-15)


def test_r_svd_diagonal_is_a_sorted_permutation(oracle):
    d = np.array([0.5, 3.0, 2.0, 7.0, 1.0])
    sig, S, st = oracle.r_svd(np.diag(d))
    assert st == 0
    np.testing.assert_array_equal(sig, np.sort(d)[::-1])
    order = np.argsort(-d)
    np.testing.assert_array_equal(np.abs(S), np.abs(np.diag(d)[order]))


@pytest.mark.parametrize("m,n", [(1, 1), (40, 7), (3000, 50), (500, 101)])
def test_r_svd_matches_lapack(oracle, m, n):
    # sigma equals LAPACK's (a different algorithm); Sigma V' = U' R with U
    # orthogonal, so (Sigma V')' (Sigma V') = R'R and the rows are orthogonal
    # with norms sigma; rows of well-separated sigma equal LAPACK's up to sign
    X = synth.random_nonneg(m, n, seed=m + n, dtype=np.float64)
    R = oracle.qr_r(X)
    sig, S, st = oracle.r_svd(R)
    assert st == 0
    U, sl, Vt = np.linalg.svd(R)
    np.testing.assert_allclose(sig, sl, rtol=0, atol=1e-12 * sl[0])
    G = R.T @ R
    assert np.linalg.norm(S.T @ S - G) <= 1e-12 * np.linalg.norm(G)
    D = S @ S.T
    assert np.max(np.abs(D - np.diag(np.diag(D)))) <= 1e-12 * sl[0] ** 2
    for i in range(n):
        gaps = [abs(sl[i] - sl[j]) for j in (i - 1, i + 1) if 0 <= j < n]
        if min(gaps, default=sl[0]) > 1e-3 * sl[0]:
            ref = sl[i] * Vt[i]
            s = np.sign(S[i] @ ref)
            np.testing.assert_allclose(s * S[i], ref, rtol=0, atol=1e-9 * sl[0])


def test_r_svd_rank_deficient(oracle):
    X, P = synth.planted_separable(5000, 20, 4, seed=14, dtype=np.float64)
    sig, S, st = oracle.r_svd(oracle.qr_r(X))
    assert st == 0
    assert np.all(sig[4:] <= 1e-10 * sig[0])
