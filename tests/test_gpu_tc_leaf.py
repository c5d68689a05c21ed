"""Parity of the tensor-core (TF32X3) pass against the FP64 oracle, through the C ABI.

The TF32X3 pass factors each 128-row tile in compact-WY form with the
trailing updates and the projection on tcgen05 (three-pass TF32 products,
FP32 accumulation).  It is held to the same bounds as the binary32 pass:

  R      : ||R_gpu - R_orc||_F / ||R_orc||_F <= 1e-5
  colsum : relative 1e-6
  GX     : |GX_gpu - GX_orc| <= 2e-6 * (|G|^T |X|) elementwise

The TF32 form (MRNMF_PREC_TF32) runs the same leaf with one TF32 product in
place of three: its operands keep 10-bit mantissas, so it is held to its own
stated bounds.  R's are about three times the largest error measured on
GB300 (4.8e-4 to 6.3e-4 on uniform X, 1.4e-3 with 10^U(0,3) column scaling).
GX's follows from the arithmetic: truncating each operand to TF32 moves it
by less than 2^-10 of itself, so each product is within 2^-9 of the exact
one, and the binary32 sums add the 2e-6 of the other forms:

  R      : relative Frobenius 2e-3 (uniform X), 5e-3 (10^U(0,3) columns)
  colsum : relative 1e-6 (summed from the same binary32 values)
  GX     : (2^-9 + 2e-6) * (|G|^T |X|) elementwise
"""
import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R_TOL = 1e-5
R_TOL_TF32 = 2e-3
R_TOL_TF32_SCALED = 5e-3
GX_TOL_TF32 = 2.0 ** -9 + 2e-6


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


def gx_bound(X, k, seed, row0=0):
    import oracle as orc
    G = orc.gauss_matrix(seed, row0, X.shape[0], k)
    return np.abs(G).T @ np.abs(X.astype(np.float64))


# one tile, a ragged tile, several tiles per stream with a ragged tail, every
# panel count (n = 17..32: 2 panels, 33..48: 3, 49..64: 4, up to 8 at n = 128),
# both tensor-memory maps (n <= 64 and 64 < n <= 128)
SHAPES = [(17, 17), (100, 20), (129, 24), (4099, 20), (20011, 30), (5000, 32), (3001, 33), (12345, 50),
          (9999, 48), (5000, 64), (128 * 152 * 2 + 77, 40), (300000, 50), (3001, 65), (40000, 100),
          (7000, 127), (20000, 128), (5000, 129), (3000, 150), (20000, 200), (4000, 256)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_tsqr_tf32x3_matches_oracle(h, oracle, m, n):
    X = synth.random_nonneg(m, n, seed=7 * m + n)
    R, cs = h.tsqr_r(dev(X), prec="tf32x3")
    h.sync()
    X64 = X.astype(np.float64)
    Ro = oracle.qr_r(X64)
    Rg = host(R)
    assert np.all(np.tril(Rg, -1) == 0) and np.all(np.diag(Rg) >= 0)
    assert rel_fro(Rg, Ro) <= R_TOL
    np.testing.assert_allclose(host(cs), oracle.colsum(X64), rtol=1e-6)


@pytest.mark.parametrize("m,n,k", [(20011, 30, 12), (9001, 50, 20), (4099, 64, 31), (50000, 40, 1), (777, 18, 15),
                                   (4096, 36, 16), (3000, 40, 32), (20000, 100, 40), (5000, 128, 48), (3000, 70, 17),
                                   (20000, 200, 40), (3000, 256, 48), (1000, 140, 5)])
def test_fused_tf32x3_matches_oracle(h, oracle, m, n, k):
    X = synth.random_nonneg(m, n, seed=3 + n + k)
    R, cs, GX = h.tsqr_gp(dev(X), k, seed=99, prec="tf32x3")
    h.sync()
    X64 = X.astype(np.float64)
    assert rel_fro(host(R), oracle.qr_r(X64)) <= R_TOL
    GXo = oracle.gauss_project(X64, k, 99)
    assert np.all(np.abs(host(GX) - GXo) <= 2e-6 * gx_bound(X, k, 99) + 1e-12)
    np.testing.assert_allclose(host(cs), oracle.colsum(X64), rtol=1e-6)


@pytest.mark.parametrize("m,n,r", [(200000, 50, 10), (60000, 200, 20)])
def test_tf32x3_ill_conditioned(h, oracle, m, n, r):
    # column scaling 10^U(0,6) (the recipe of the 1e8 x 200 workload): per-column
    # relative error bounded as for binary32
    X, P = synth.planted_separable(m, n, r, seed=1402003, noise=1e-3, decades=6.0)
    R, _ = h.tsqr_r(dev(X), prec="tf32x3")
    h.sync()
    Ro = oracle.qr_r(X.astype(np.float64))
    Rg = host(R)
    assert rel_fro(Rg, Ro) <= R_TOL
    col = np.linalg.norm(Rg - Ro, axis=0) / np.linalg.norm(Ro, axis=0)
    assert np.max(col) < 1e-4


def test_tf32x3_rank_deficient(h, oracle):
    # exact low rank (r = 5 < n = 40): R^T R = X^T X still holds, and rows
    # past the rank are at rounding level
    X, P = synth.planted_separable(30000, 40, 5, seed=8)
    R, _ = h.tsqr_r(dev(X), prec="tf32x3")
    h.sync()
    Rg = host(R).astype(np.float64)
    X64 = X.astype(np.float64)
    G = X64.T @ X64
    assert np.linalg.norm(Rg.T @ Rg - G) / np.linalg.norm(G) <= 2 * R_TOL
    assert np.linalg.norm(Rg[5:]) <= 1e-4 * np.linalg.norm(Rg)


def test_tf32x3_streaming(h, oracle):
    X = synth.random_nonneg(50000, 36, seed=17)
    h.stream_begin(36, prec="tf32x3", k=8, seed=3)
    for a, b in [(0, 1), (1, 4000), (4000, 4001), (4001, 33333), (33333, 50000)]:
        h.stream_push(dev(X[a:b]))
    R, cs, GX = h.stream_end(36, k=8)
    h.sync()
    X64 = X.astype(np.float64)
    assert rel_fro(host(R), oracle.qr_r(X64)) <= R_TOL
    np.testing.assert_allclose(host(cs), oracle.colsum(X64), rtol=1e-6)
    GXo = oracle.gauss_project(X64, 8, 3)
    assert np.all(np.abs(host(GX) - GXo) <= 2e-6 * gx_bound(X, 8, 3) + 1e-12)


def test_tf32x3_strided_rows(h, oracle):
    W = synth.random_nonneg(3000, 60, seed=5)
    Xd = dev(W)[:, 3:53]
    R, _ = h.tsqr_r(Xd, prec="tf32x3")
    h.sync()
    assert rel_fro(host(R), oracle.qr_r(W[:, 3:53].astype(np.float64))) <= R_TOL


def test_tf32x3_bad_input_is_reported(h):
    from paper_1402_6964_gb300 import mrnmf
    X = synth.random_nonneg(5000, 30, seed=1)
    for mutate in ("neg", "nan"):
        Y = X.copy()
        if mutate == "neg":
            Y[1234, 4] = -1e-3
        else:
            Y[77, 29] = np.nan
        h.tsqr_r(dev(Y), prec="tf32x3")
        with pytest.raises(mrnmf.MrnmfError) as e:
            h.sync()
        assert e.value.status == mrnmf.ERR_BAD_INPUT
    h.tsqr_r(dev(X), prec="tf32x3")
    h.sync()


def test_tf32x3_rejects_unsupported_shape(h):
    # the tensor-core form covers 16 < n <= 256, with k <= 32 for n <= 64 and k <= 48 above
    from paper_1402_6964_gb300 import mrnmf
    for prec in ("tf32x3", "tf32"):
        X = synth.random_nonneg(1000, 10, seed=2)
        with pytest.raises(mrnmf.MrnmfError) as e:
            h.tsqr_r(dev(X), prec=prec)
        assert e.value.status == mrnmf.ERR_INVALID_ARG
        for n, k in [(50, 33), (100, 49)]:
            X = synth.random_nonneg(1000, n, seed=2)
            with pytest.raises(mrnmf.MrnmfError) as e:
                h.tsqr_gp(dev(X), k, seed=1, prec=prec)
            assert e.value.status == mrnmf.ERR_INVALID_ARG


@pytest.mark.parametrize("m,n,k", [(200_000, 50, 0), (200_000, 50, 20), (50_000, 20, 8), (60_000, 200, 40),
                                   (40_000, 256, 0), (3001, 65, 17), (129, 24, 0)])
def test_tsqr_tf32_single_product_within_its_bound(h, oracle, m, n, k):
    X = synth.random_nonneg(m, n, seed=7 + n)
    X64 = X.astype(np.float64)
    if k:
        R, cs, GX = h.tsqr_gp(dev(X), k, seed=3, prec="tf32")
    else:
        R, cs = h.tsqr_r(dev(X), prec="tf32")
    h.sync()
    Rg = host(R)
    assert np.all(np.tril(Rg, -1) == 0) and np.all(np.diag(Rg) >= 0)
    err = rel_fro(Rg, oracle.qr_r(X64))
    assert err <= R_TOL_TF32, err
    # the single product is a different form: its error is far from the three-product form's
    assert err > 1e-5
    np.testing.assert_allclose(host(cs), oracle.colsum(X64), rtol=1e-6)
    if k:
        GXo = oracle.gauss_project(X64, k, 3)
        assert np.all(np.abs(host(GX) - GXo) <= GX_TOL_TF32 * gx_bound(X, k, 3) + 1e-12)


def test_tsqr_tf32_scaled_columns(h, oracle):
    X, _ = synth.planted_separable(100_000, 100, 10, seed=107, noise=1e-3, decades=3.0)
    R, _ = h.tsqr_r(dev(X), prec="tf32")
    h.sync()
    assert rel_fro(host(R), oracle.qr_r(X.astype(np.float64))) <= R_TOL_TF32_SCALED
