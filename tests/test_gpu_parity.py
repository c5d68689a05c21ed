"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (stated once, used below):
  R, FP32 pass : ||R_gpu - R_orc||_F / ||R_orc||_F <= 1e-5  (target fixed for the FP32 form)
  R, FP64 pass : <= 1e-12
  R columns    : on the 10^U(0,6)-scaled recipe, every column within relative 1e-4
  colsum       : relative 1e-6 (FP32 pass; binary32 tile sums, binary64 across tiles)
  GX           : |GX_gpu - GX_orc| <= 2e-6 * (|G|^T |X|) elementwise, the natural bound of
                 a binary32 sum of products (G drawn in binary32 on the device)
  H, residual  : relative 1e-4 when K matches; 1e-9 on identical inputs
  K            : bit-exact at every pick whose relative gap exceeds the margin
                 (100x the pass's R error); smaller gaps are tie-ambiguous and only the
                 validity of the pick is checked.
"""
import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R_TOL_FP32 = 1e-5
# largest per-column relative error of R on the ill-conditioned recipe
# (10^U(0,6) column scaling): measured 2.3e-5 at 1e6 rows, 5.5e-5 at 6e4 rows
COL_TOL_ILLCOND = 1e-4


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_6964_gb300 import build, mrnmf
    build.build()
    hd = mrnmf.Handle()
    yield hd
    hd.close()


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def compare_K(Kg, Ko, gap, margin, n=None):
    """Margin rule: picks must agree at every step whose oracle gap (relative
    margin between the best and second-best score) exceeds `margin`.  At a
    smaller gap the two orders may legitimately differ; from the first such
    divergence on the sequences are not comparable pick by pick, so what
    remains is checked for validity: every pick is a distinct column index in
    [0, n).  Returns the number of leading picks that agree."""
    Kg = [int(v) for v in Kg]
    assert len(set(Kg)) == len(Kg), f"repeated pick in {Kg}"
    if n is not None:
        assert all(0 <= v < n for v in Kg), f"pick out of range in {Kg}"
    for t in range(len(Ko)):
        if Kg[t] != Ko[t]:
            assert gap[t] < margin, f"pick {t}: gpu {Kg[t]} vs oracle {Ko[t]} (gap {gap[t]:.3g} > {margin:.3g})"
            return t
    return len(Ko)


def k_margin(Rg, Ro):
    """100x the measured relative error of the pass's R (scores are quadratic
    in R, so a relative R error e moves them by about 2e)."""
    return max(100.0 * rel_fro(Rg, Ro), 1e-12)


# --------------------------------------------------------------------- R

SHAPES = [(1, 1), (5, 5), (17, 3), (33, 32), (1000, 1), (1000, 7), (4099, 20), (12345, 50),
          (5000, 64), (3001, 65), (20000, 128), (7001, 200), (3000, 256)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_tsqr_fp32_matches_oracle(h, oracle, m, n):
    X = synth.random_nonneg(m, n, seed=m * 1000 + n)
    R, cs = h.tsqr_r(dev(X), prec="fp32")
    h.sync()
    Ro = oracle.qr_r(X.astype(np.float64))
    Rg = host(R)
    assert np.all(np.tril(Rg, -1) == 0) and np.all(np.diag(Rg) >= 0)
    assert rel_fro(Rg, Ro) <= R_TOL_FP32
    np.testing.assert_allclose(host(cs), oracle.colsum(X.astype(np.float64)), rtol=1e-6)


@pytest.mark.parametrize("m,n", [(1, 1), (37, 20), (20000, 20), (9999, 64), (4000, 128)])
def test_tsqr_fp64_matches_oracle(h, oracle, m, n):
    X = synth.random_nonneg(m, n, seed=77 + n, dtype=np.float64)
    R, cs = h.tsqr_r(dev(X), prec="fp64")
    h.sync()
    assert rel_fro(host(R), oracle.qr_r(X)) <= 1e-12
    np.testing.assert_allclose(host(cs), oracle.colsum(X), rtol=1e-13)


def test_tsqr_strided_rows(h, oracle):
    # ldx > n: X is a column slice of a wider row-major array
    W = synth.random_nonneg(3000, 40, seed=5)
    Xd = dev(W)[:, 3:33]
    R, _ = h.tsqr_r(Xd, prec="fp32")
    h.sync()
    assert rel_fro(host(R), oracle.qr_r(W[:, 3:33].astype(np.float64))) <= R_TOL_FP32


def test_tsqr_ill_conditioned(h, oracle):
    # column scaling 10^U(0,6) (cond ~ 1e6): R per column relative error stays
    # at the FP32 backward-error level scaled by each column's size
    X, P = synth.planted_separable(200000, 40, 8, seed=1402003, noise=1e-3, decades=6.0)
    R, _ = h.tsqr_r(dev(X), prec="fp32")
    h.sync()
    Ro = oracle.qr_r(X.astype(np.float64))
    Rg = host(R)
    assert rel_fro(Rg, Ro) <= R_TOL_FP32
    col = np.linalg.norm(Rg - Ro, axis=0) / np.linalg.norm(Ro, axis=0)
    assert np.max(col) < COL_TOL_ILLCOND


def test_fused_ill_conditioned_n200(h, oracle):
    # the 1e8 x 200 workload's recipe (r = 20, 10^U(0,6) column scaling, k = 40)
    # at 60,000 rows, through the pipelined leaf and the fan-in-2 tree: R, the
    # column sums and GX against the oracle on the same rows
    X, P = synth.planted_separable(60000, 200, 20, seed=1402002, noise=1e-3, decades=6.0)
    R, cs, GX = h.tsqr_gp(dev(X), 40, seed=1402002)
    h.sync()
    X64 = X.astype(np.float64)
    Ro = oracle.qr_r(X64)
    Rg = host(R)
    assert rel_fro(Rg, Ro) <= R_TOL_FP32
    col = np.linalg.norm(Rg - Ro, axis=0) / np.linalg.norm(Ro, axis=0)
    assert np.max(col) < COL_TOL_ILLCOND
    np.testing.assert_allclose(host(cs), oracle.colsum(X64), rtol=1e-6)
    GXo = oracle.gauss_project(X64, 40, 1402002)
    assert np.all(np.abs(host(GX) - GXo) <= 2e-6 * _gx_bound(X, 40, 1402002) + 1e-12)


def test_bad_input_is_reported(h):
    from paper_1402_6964_gb300 import mrnmf
    X = synth.random_nonneg(500, 6, seed=1)
    for mutate in ("neg", "nan", "zerocol"):
        Y = X.copy()
        if mutate == "neg":
            Y[123, 4] = -1e-3
        elif mutate == "nan":
            Y[77, 2] = np.nan
        else:
            Y[:, 3] = 0.0
        h.tsqr_r(dev(Y), prec="fp32")
        with pytest.raises(mrnmf.MrnmfError) as e:
            h.sync()
        assert e.value.status == mrnmf.ERR_BAD_INPUT
    # the handle stays usable afterwards
    h.tsqr_r(dev(X), prec="fp32")
    h.sync()


# -------------------------------------------------------------------- GX

def _gx_bound(X, k, seed, row0=0):
    import oracle as orc
    G = orc.gauss_matrix(seed, row0, X.shape[0], k)
    return np.abs(G).T @ np.abs(X.astype(np.float64))


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (1000, 7, 3), (4099, 20, 10), (30011, 50, 20), (5000, 128, 64)])
def test_gauss_project_matches_oracle(h, oracle, m, n, k):
    X = synth.random_nonneg(m, n, seed=m + n + k)
    GX, cs = h.gauss_project(dev(X), k, seed=1234567, row_offset=0)
    h.sync()
    GXo = oracle.gauss_project(X.astype(np.float64), k, 1234567)
    assert np.all(np.abs(host(GX) - GXo) <= 2e-6 * _gx_bound(X, k, 1234567) + 1e-12)
    np.testing.assert_allclose(host(cs), oracle.colsum(X.astype(np.float64)), rtol=1e-6)


def test_gauss_project_row_offset(h, oracle):
    X = synth.random_nonneg(3000, 9, seed=9)
    GX, _ = h.gauss_project(dev(X), 6, seed=42, row_offset=10_000_000_000)
    h.sync()
    GXo = oracle.gauss_project(X.astype(np.float64), 6, 42, row0=10_000_000_000)
    assert np.all(np.abs(host(GX) - GXo) <= 2e-6 * _gx_bound(X, 6, 42, 10_000_000_000) + 1e-12)


@pytest.mark.parametrize("m,n,k", [(20011, 30, 12), (9001, 50, 20), (20011, 100, 40), (4003, 200, 40),
                                   (2000, 65, 17), (5000, 100, 64), (3001, 256, 64), (777, 224, 1)])
def test_fused_pass_matches_separate(h, oracle, m, n, k):
    # Sec. 3.5: TSQR and GP in one pass give what the two separate passes give
    X = synth.random_nonneg(m, n, seed=3 + n)
    R, cs, GX = h.tsqr_gp(dev(X), k, seed=99, prec="fp32")
    h.sync()
    Ro = oracle.qr_r(X.astype(np.float64))
    assert rel_fro(host(R), Ro) <= R_TOL_FP32
    GXo = oracle.gauss_project(X.astype(np.float64), k, 99)
    assert np.all(np.abs(host(GX) - GXo) <= 2e-6 * _gx_bound(X, k, 99) + 1e-12)
    np.testing.assert_allclose(host(cs), oracle.colsum(X.astype(np.float64)), rtol=1e-6)


# ---------------------------------------------- the n-by-n step, same inputs

@pytest.fixture(scope="module")
def reduced(oracle):
    X, P = synth.planted_separable(60000, 48, 9, seed=21, noise=1e-3)
    X64 = X.astype(np.float64)
    return X, P, oracle.qr_r(X64), oracle.colsum(X64), oracle.gauss_project(X64, 18, 5)


def test_spa_same_input(h, oracle, reduced):
    X, P, Ro, so, GXo = reduced
    K, gap = h.select_extreme("spa", R=dev(Ro), colsum=dev(so), r=9)
    h.sync()
    Ko, go = oracle.spa(Ro, so, 9)
    assert list(host(K)) == list(Ko)
    np.testing.assert_allclose(host(gap), go, rtol=1e-9, atol=1e-12)


def test_xray_same_input(h, oracle, reduced):
    X, P, Ro, so, GXo = reduced
    K, gap = h.select_extreme("xray", R=dev(Ro), r=9)
    h.sync()
    Ko, go, st = oracle.xray(Ro, 9)
    assert list(host(K)) == list(Ko)
    np.testing.assert_allclose(host(gap), go, rtol=1e-8, atol=1e-12)


def test_gp_same_input(h, oracle, reduced):
    X, P, Ro, so, GXo = reduced
    K, gap = h.select_extreme("gp", colsum=dev(so), GX=dev(GXo), r=9)
    h.sync()
    Ko, cand, cg = oracle.gp_select(GXo, so, 9)
    assert list(host(K)) == list(Ko)
    np.testing.assert_allclose(host(gap), cg[:9], rtol=1e-9, atol=1e-12)


def test_nnls_residual_same_input(h, oracle, reduced):
    X, P, Ro, so, GXo = reduced
    K = P.K
    H = h.nnls_h(dev(Ro), dev(K.astype(np.int32)))
    out = h.residual(dev(Ro), dev(K.astype(np.int32)), H)
    h.sync()
    Ho, st = oracle.nnls_h(Ro, K)
    assert st == 0
    np.testing.assert_allclose(host(H), Ho, rtol=1e-9, atol=1e-11)
    ab, rel = oracle.residual(Ro, K, Ho)
    o = host(out)
    assert o[0] == pytest.approx(ab, rel=1e-9) and o[1] == pytest.approx(rel, rel=1e-9)


def test_nnls_repeated_column(h, oracle):
    # a repeated index makes R(:,K) singular; Lawson-Hanson never activates the
    # copy (its dual equals the original's, which is zero at the optimum), so
    # the fit equals the one with the duplicate removed
    X = synth.random_nonneg(400, 10, seed=8).astype(np.float64)
    Ro = oracle.qr_r(X)
    Kd = dev(np.array([2, 2, 5], np.int32))
    H = h.nnls_h(dev(Ro), Kd)
    out = h.residual(dev(Ro), Kd, H)
    h.sync()
    Ho, st = oracle.nnls_h(Ro, np.array([2, 5], np.int32))
    ab, rel = oracle.residual(Ro, np.array([2, 5], np.int32), Ho)
    assert host(out)[0] == pytest.approx(ab, rel=1e-9)
    Hg = host(H)
    np.testing.assert_allclose(Hg[0] + Hg[1], Ho[0], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(Hg[2], Ho[1], rtol=1e-9, atol=1e-12)


# ----------------------------------------------------------- end to end

def test_exact_separable_fp64_end_to_end(h, oracle):
    # 20000 x 20, r = 5, FP64: K exact, zero residual (Sec. 4)
    w = synth.WORKLOADS["exact_fp64"]
    X, P = synth.workload_matrix(w)
    R, cs = h.tsqr_r(dev(X), prec="fp64")
    K, gap = h.select_extreme("spa", R=R, colsum=cs, r=w.r)
    H = h.nnls_h(R, K)
    out = h.residual(R, K, H)
    h.sync()
    Rg = host(R)
    np.testing.assert_allclose(Rg.T @ Rg, X.T @ X, rtol=1e-11, atol=1e-9 * np.abs(X.T @ X).max())
    assert sorted(host(K)) == list(P.K)
    Ko, _ = oracle.spa(oracle.qr_r(X), oracle.colsum(X), w.r)
    assert list(host(K)) == list(Ko)
    assert host(out)[1] < 1e-20
    order = np.argsort(host(K))
    np.testing.assert_allclose(host(H)[order], P.H_true, atol=1e-9)


@pytest.mark.parametrize("method", ["spa", "xray", "gp"])
def test_near_separable_end_to_end(h, oracle, method):
    # near-separable FP32 (sigma = 1e-3), 2e5 x 50, r = 10, k = 20
    X, P = synth.planted_separable(200000, 50, 10, seed=1402002, noise=1e-3)
    X64 = X.astype(np.float64)
    R, cs, GX = h.tsqr_gp(dev(X), 20, seed=7, prec="fp32")
    K, gap = h.select_extreme(method, R=R, colsum=cs, GX=GX if method == "gp" else None, r=10)
    H = h.nnls_h(R, K)
    out = h.residual(R, K, H)
    h.sync()
    Ro = oracle.qr_r(X64)
    so = oracle.colsum(X64)
    if method == "spa":
        Ko, go = oracle.spa(Ro, so, 10)
    elif method == "xray":
        Ko, go, _ = oracle.xray(Ro, 10)
    else:
        Ko, cand, go = oracle.gp_select(oracle.gauss_project(X64, 20, 7), so, 10)
    Kg = host(K)
    t = compare_K(Kg, Ko, go, k_margin(host(R), Ro), n=50)
    if t == 10:
        Ho, _ = oracle.nnls_h(Ro, Ko)
        assert rel_fro(host(H), Ho) <= 1e-4
        ab, rel = oracle.residual(Ro, Ko, Ho)
        assert host(out)[0] == pytest.approx(ab, rel=1e-4)
    if method != "xray":
        assert sorted(Kg) == list(P.K)  # SPA and GP recover the planted columns (Sec. 4)


def test_streaming_matches_one_shot(h, oracle):
    X = synth.random_nonneg(50000, 24, seed=17)
    h.stream_begin(24, k=8, seed=3)
    for a, b in [(0, 1), (1, 4000), (4000, 4001), (4001, 33333), (33333, 50000)]:
        h.stream_push(dev(X[a:b]))
    R, cs, GX = h.stream_end(24, k=8)
    h.sync()
    X64 = X.astype(np.float64)
    assert rel_fro(host(R), oracle.qr_r(X64)) <= R_TOL_FP32
    np.testing.assert_allclose(host(cs), oracle.colsum(X64), rtol=1e-6)
    GXo = oracle.gauss_project(X64, 8, 3)
    assert np.all(np.abs(host(GX) - GXo) <= 2e-6 * _gx_bound(X, 8, 3) + 1e-12)


def test_factorize_host(h, oracle):
    X, P = synth.planted_separable(100000, 30, 6, seed=44, noise=1e-3)
    K, H, res, R = h.factorize_host(X, 6, method="spa", want_R=True)
    X64 = X.astype(np.float64)
    Ro = oracle.qr_r(X64)
    assert rel_fro(R, Ro) <= R_TOL_FP32
    Ko, go = oracle.spa(Ro, oracle.colsum(X64), 6)
    if compare_K(K, Ko, go, k_margin(R, Ro), n=30) == 6:
        Ho, _ = oracle.nnls_h(Ro, Ko)
        assert rel_fro(H, Ho) <= 1e-4
    assert sorted(K) == list(P.K)


def test_full_size_near_separable(h, oracle):
    """1e7 x 50 FP32 (the benchmarked workload) in bench.py's launch
    configuration: R by the Gram identity R^T R = X^T X and against the unique
    R = chol(X^T X)^T (a library route), colsum, the fused pass's GX against the
    oracle's row-by-row G^T X, and SPA's K against the oracle's SPA on that R."""
    w = synth.WORKLOADS["near_sep_1e7x50"]
    X, P = synth.workload_matrix(w)
    R, cs, GX = h.tsqr_gp(dev(X), w.k, seed=w.seed, prec="auto")
    K, gap = h.select_extreme("spa", R=R, colsum=cs, r=w.r)
    h.sync()
    Rg = host(R)
    X64 = X.astype(np.float64)
    G = X64.T @ X64
    assert np.linalg.norm(Rg.T @ Rg - G) / np.linalg.norm(G) <= 2 * R_TOL_FP32
    Rc = np.linalg.cholesky(G).T
    assert rel_fro(Rg, Rc) <= R_TOL_FP32
    np.testing.assert_allclose(host(cs), X64.sum(0), rtol=1e-6)
    GXo = oracle.gauss_project(X64, w.k, w.seed)
    assert np.all(np.abs(host(GX) - GXo) <= 2e-6 * _gx_bound(X, w.k, w.seed) + 1e-12)
    Ko, go = oracle.spa(Rc, X64.sum(0), w.r)
    if compare_K(host(K), Ko, go, k_margin(Rg, Rc), n=w.n) == w.r:
        H = h.nnls_h(R, K)
        out = h.residual(R, K, H)
        h.sync()
        Ho, _ = oracle.nnls_h(Rc, Ko)
        assert rel_fro(host(H), Ho) <= 1e-4
        ab, rel = oracle.residual(Rc, Ko, Ho)
        assert host(out)[0] == pytest.approx(ab, rel=1e-4)
    assert sorted(host(K)) == list(P.K)


@pytest.mark.parametrize("method", ["spa", "xray", "gp"])
def test_rank_sweep(h, oracle, reduced, method):
    # Sec. 2.4 / Sec. 5: residual for every r <= r_max from one R, against the
    # oracle's NNLS + residual on the oracle's nested picks (same inputs)
    X, P, Ro, so, GXo = reduced
    r_max = 12
    if method == "gp":  # GP only ever proposes extreme points: sweep up to its candidate count
        r_max = min(r_max, len(oracle.gp_select(GXo, so, 1)[1]))
    K, curve = h.rank_sweep(method, R=dev(Ro), colsum=dev(so), GX=dev(GXo) if method == "gp" else None, r_max=r_max)
    h.sync()
    if method == "spa":
        Ko, _ = oracle.spa(Ro, so, r_max)
    elif method == "xray":
        Ko, _, _ = oracle.xray(Ro, r_max)
    else:
        Ko, _, _ = oracle.gp_select(GXo, so, r_max)
    assert list(host(K)) == list(Ko)
    cv = host(curve)
    for r in range(1, r_max + 1):
        Hr, _ = oracle.nnls_h(Ro, Ko[:r])
        ab, rel = oracle.residual(Ro, Ko[:r], Hr)
        assert cv[r - 1, 0] == pytest.approx(ab, rel=1e-8, abs=1e-12)
        assert cv[r - 1, 1] == pytest.approx(rel, rel=1e-8, abs=1e-20)
    # the curve drops to the noise floor at the planted rank (9) for SPA and GP
    if method != "xray" and r_max >= 9:
        assert cv[8, 1] < 1e-4 * cv[0, 1]


# ------------------------------- the 1e8 x 200 recipe, K / H / residual

@pytest.fixture(scope="module")
def illcond200(oracle):
    """The ill-conditioned workload's recipe (n = 200, r = 20, 10^U(0,6)
    column scaling, sigma = 1e-3, k = 40) at 200,000 rows, with the oracle's
    R, column sums and GX of the same rows."""
    w = synth.WORKLOADS["illcond_1e8x200"]
    X, P = synth.workload_matrix(w, m=200_000)
    X64 = X.astype(np.float64)
    return w, X, P, oracle.qr_r(X64), oracle.colsum(X64), oracle.gauss_project(X64, w.k, w.seed)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
@pytest.mark.parametrize("method", ["spa", "xray", "gp"])
def test_illcond_n200_select_nnls_residual(h, oracle, illcond200, method, prec):
    """K (margin rule), H and the residual against the oracle on the
    1e8 x 200 recipe at 2e5 rows, through the fused pass in each arithmetic
    form.  SPA recovers the planted columns; GP's candidates are planted
    columns, and when its k = 40 rows propose fewer than r distinct columns
    the device reports it (as the oracle finds) and the step runs on those."""
    from paper_1402_6964_gb300 import mrnmf
    w, X, P, Ro, so, GXo = illcond200
    R, cs, GX = h.tsqr_gp(dev(X), w.k, seed=w.seed, prec=prec)
    h.sync()
    Rg = host(R)
    assert rel_fro(Rg, Ro) <= R_TOL_FP32
    col = np.linalg.norm(Rg - Ro, axis=0) / np.linalg.norm(Ro, axis=0)
    assert np.max(col) < COL_TOL_ILLCOND
    r = w.r
    if method == "gp":
        cand = oracle.gp_select(GXo, so, 1)[1]
        if len(cand) < r:
            h.select_extreme("gp", colsum=cs, GX=GX, r=r)
            with pytest.raises(mrnmf.MrnmfError) as e:
                h.sync()
            assert e.value.status == mrnmf.ERR_RANK_DEFICIENT
            r = len(cand)
    K, gap = h.select_extreme(method, R=R, colsum=cs, GX=GX if method == "gp" else None, r=r)
    H = h.nnls_h(R, K)
    out = h.residual(R, K, H)
    h.sync()
    if method == "spa":
        Ko, go = oracle.spa(Ro, so, r)
    elif method == "xray":
        Ko, go, _ = oracle.xray(Ro, r)
    else:
        Ko, cand, go = oracle.gp_select(GXo, so, r)
    Kg = host(K)
    t = compare_K(Kg, Ko, go, k_margin(Rg, Ro), n=w.n)
    if t == r:
        Ho, _ = oracle.nnls_h(Ro, Ko)
        assert rel_fro(host(H), Ho) <= 1e-4
        ab, rel = oracle.residual(Ro, Ko, Ho)
        o = host(out)
        assert o[0] == pytest.approx(ab, rel=1e-4) and o[1] == pytest.approx(rel, rel=1e-4)
    if method == "spa":
        assert sorted(Kg) == list(P.K)
    elif method == "gp":
        assert set(int(v) for v in Kg) <= set(int(v) for v in P.K)


def test_xray_exact_data_contains_planted(h, oracle):
    """Sec. 4: on exact separable data greedy XRAY finds every planted column
    within r + 1 picks (the paper needed 21 picks for 20 columns); the GPU's
    r + 1 picks equal the oracle's."""
    w = synth.WORKLOADS["exact_fp64"]
    X, P = synth.workload_matrix(w)
    R, cs = h.tsqr_r(dev(X), prec="fp64")
    K, gap = h.select_extreme("xray", R=R, r=w.r + 1)
    h.sync()
    Kg = [int(v) for v in host(K)]
    assert set(P.K) <= set(Kg)
    Ko, go, _ = oracle.xray(oracle.qr_r(X), w.r + 1)
    compare_K(Kg, Ko, go, k_margin(host(R), oracle.qr_r(X)), n=w.n)


def test_binary64_tree_matches_oracle(oracle):
    """The binary64 tree over binary32 leaf triangles (MRNMF_TREE64=1, read once
    per process, so the pass runs in a child process): R against the oracle on
    the ill-conditioned recipe at n = 200 (pipelined leaf) and at n = 50 (warp
    leaf, four streams folded per CTA), both within the FP32 bounds."""
    import os
    import subprocess
    import sys
    code = (
        "import sys, numpy as np, torch\n"
        "sys.path.insert(0, %r)\n"
        "from paper_1402_6964_gb300 import mrnmf, synth\n"
        "h = mrnmf.Handle()\n"
        "for m, n, r, seed in [(60000, 200, 20, 1402003), (300000, 50, 10, 1402002)]:\n"
        "    X, _ = synth.planted_separable(m, n, r, seed=seed, noise=1e-3, decades=6.0)\n"
        "    R, _ = h.tsqr_r(torch.from_numpy(X).cuda(), prec='fp32'); h.sync()\n"
        "    np.save('/tmp/tree64_%%d.npy' %% n, R.cpu().numpy())\n"
    ) % os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, MRNMF_TREE64="1")
    subprocess.run([sys.executable, "-c", code], env=env, check=True, timeout=600)
    for m, n, r, seed in [(60000, 200, 20, 1402003), (300000, 50, 10, 1402002)]:
        X, _ = synth.planted_separable(m, n, r, seed=seed, noise=1e-3, decades=6.0)
        Ro = oracle.qr_r(X.astype(np.float64))
        Rg = np.load("/tmp/tree64_%d.npy" % n)
        assert np.all(np.tril(Rg, -1) == 0) and np.all(np.diag(Rg) >= 0)
        assert rel_fro(Rg, Ro) <= R_TOL_FP32
        col = np.linalg.norm(Rg - Ro, axis=0) / np.linalg.norm(Ro, axis=0)
        assert np.max(col) < COL_TOL_ILLCOND


def test_tuned_stream_counts_match_oracle(h, oracle, tmp_path):
    """Tuning-table settings change only the amount of parallel work: with far
    fewer and with more row streams than the default (pass lines), and with
    other batch waves, R still matches the oracle within the FP32 bound."""
    from paper_1402_6964_gb300 import mrnmf
    cases = [(200_000, 50), (60_000, 200), (30_000, 12)]
    try:
        for factor in (0.125, 4.0):
            path = tmp_path / f"t{factor}.txt"
            path.write_text(f"pass 1 256 0 64 {factor}\nbatch 1 1\nbatch 2 4\nbatch 3 8\n")
            assert mrnmf.tune_load(str(path)) == mrnmf.OK
            for m, n in cases:
                X = synth.random_nonneg(m, n, seed=m + n)
                R, cs = h.tsqr_r(dev(X), prec="fp32")
                h.sync()
                assert rel_fro(host(R), oracle.qr_r(X.astype(np.float64))) <= R_TOL_FP32, (factor, m, n)
            Xs = [synth.random_nonneg(m, n, seed=m * n) for m, n in [(50_000, 20), (40_000, 60), (30_000, 100)]]
            outs = h.tsqr_r_batched([dev(X) for X in Xs])
            h.sync()
            for X, (R, cs) in zip(Xs, outs):
                assert rel_fro(host(R), oracle.qr_r(X.astype(np.float64))) <= R_TOL_FP32
    finally:
        mrnmf.tune_load(None)


@pytest.mark.parametrize("n,k,rows", [(30, 0, 128), (20, 12, 128), (50, 0, 64), (50, 20, 64), (60, 20, 64),
                                      (64, 0, 64)])
def test_tuned_tile_heights_match_oracle(h, oracle, tmp_path, n, k, rows):
    """A rows line changes the warp leaf's tile height; R, the column sums and
    G'X stay within the FP32 bounds of the oracle (m not a multiple of the
    height, so every stream ends on a ragged tile)."""
    from paper_1402_6964_gb300 import mrnmf
    path = tmp_path / "rows.txt"
    path.write_text(f"rows {n} {n} {k} {k} {rows}\n")
    m = 150_001
    X = synth.random_nonneg(m, n, seed=7 * n + k)
    X64 = X.astype(np.float64)
    try:
        assert mrnmf.tune_load(str(path)) == mrnmf.OK
        assert mrnmf.tune_leaf_rows(n, k) == rows
        if k:
            R, cs, GX = h.tsqr_gp(dev(X), k, seed=31, prec="fp32")
        else:
            R, cs = h.tsqr_r(dev(X), prec="fp32")
        h.sync()
    finally:
        mrnmf.tune_load(None)
    assert rel_fro(host(R), oracle.qr_r(X64)) <= R_TOL_FP32
    np.testing.assert_allclose(host(cs), oracle.colsum(X64), rtol=1e-6)
    if k:
        GXo = oracle.gauss_project(X64, k, 31)
        assert np.all(np.abs(host(GX) - GXo) <= 2e-6 * _gx_bound(X, k, 31) + 1e-12)
