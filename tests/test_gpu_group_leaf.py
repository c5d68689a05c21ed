"""The lane-group leaf (n <= 28, no projection) against the FP64 oracle.

Every binary32 pass with n <= 28 and k = 0 runs on it: a warp holds 32/S
Householder streams of S = 4, 8, 16 or 32 lanes, each on an interleaved share of
the warp's super-tiles, folded into one triangle per CTA at the end of the
launch.  Checked here, element by element against the oracle (R within the
FP32 pass tolerance, relative Frobenius 1e-5; column sums within relative
1e-6):

* every n from 1 to 16 and six widths from 17 to 28, so each group size and
  each partly filled group;
* row counts below one super-tile, at ragged multiples, and large enough for
  many tiles per stream and several binary64 flushes of the column sums;
* strided rows (ldx > n) and a base address off the 16-byte grid, which take
  the direct-load path instead of the bulk copies;
* a stream pushed in ragged chunks, where each launch continues from the
  state of the last (the CTA's triangle seeds group 0 of warp 0);
* the input check: -0 passes, a negative entry, -inf and NaN are reported;
* 10^U(0,6) column scaling, per-column error within the ill-conditioned bound.
"""
import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R_TOL_FP32 = 1e-5
CS_RTOL = 1e-6
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


def host(t):
    return t.detach().cpu().numpy()


def check(oracle, X, R, cs):
    X64 = X.astype(np.float64)
    Rg = host(R)
    assert np.all(np.tril(Rg, -1) == 0) and np.all(np.diag(Rg) >= 0)
    assert rel_fro(Rg, oracle.qr_r(X64)) <= R_TOL_FP32
    np.testing.assert_allclose(host(cs), oracle.colsum(X64), rtol=CS_RTOL)


@pytest.mark.parametrize("n", list(range(1, 17)) + [17, 18, 20, 24, 25, 28])
def test_every_width_matches_oracle(h, oracle, n):
    from paper_1402_6964_gb300 import mrnmf
    assert mrnmf.tune_leaf_rows(n, 0) in (64, 128, 256, 512)  # the group leaf's super-tile
    for m in (n, n + 1, 300, 4099, 200_003):
        X = synth.random_nonneg(m, n, seed=31 * n + m)
        R, cs = h.tsqr_r(torch.from_numpy(X).cuda(), prec="fp32")
        h.sync()
        check(oracle, X, R, cs)


@pytest.mark.parametrize("m,n", [(2_000_003, 8), (1_500_001, 13), (3_000_000, 4), (1_000_003, 25), (800_001, 28)])
def test_many_tiles_per_stream(h, oracle, m, n):
    # tens of super-tiles per stream: several binary64 flushes of the column sums
    X = synth.random_nonneg(m, n, seed=m % 1000 + n)
    R, cs = h.tsqr_r(torch.from_numpy(X).cuda(), prec="fp32")
    h.sync()
    check(oracle, X, R, cs)


@pytest.mark.parametrize("n", [3, 8, 12, 16, 25, 28])
def test_direct_load_paths(h, oracle, n):
    W = synth.random_nonneg(50_001, n + 5, seed=n)
    Xs = torch.from_numpy(W).cuda()[:, 2:2 + n]            # ldx = n + 5
    R, cs = h.tsqr_r(Xs, prec="fp32")
    h.sync()
    check(oracle, np.ascontiguousarray(W[:, 2:2 + n]), R, cs)
    flat = torch.from_numpy(synth.random_nonneg(50_001 * n + 1, 1, seed=n + 1).ravel()).cuda()
    Xo = flat[1:].view(50_001, n)                           # base 4 bytes off the 16-byte grid
    assert Xo.data_ptr() % 16 != 0
    R, cs = h.tsqr_r(Xo, prec="fp32")
    h.sync()
    check(oracle, host(Xo), R, cs)


@pytest.mark.parametrize("n", [5, 8, 16, 25])
def test_stream_in_ragged_chunks(h, oracle, n):
    X = synth.random_nonneg(700_007, n, seed=400 + n)
    Xd = torch.from_numpy(X).cuda()
    h.stream_begin(n, prec="fp32")
    a = 0
    for size in (1, 333, 65_536, 250_001, 17, 384_119):
        h.stream_push(Xd[a:a + size])
        a += size
    assert a == X.shape[0]
    R, cs, _ = h.stream_end(n)
    h.sync()
    check(oracle, X, R, cs)


def test_input_check(h, oracle):
    from paper_1402_6964_gb300 import mrnmf
    X = synth.random_nonneg(100_000, 8, seed=5)
    Y = X.copy()
    Y[::997, 3] = -0.0                                       # -0 is a nonnegative entry
    R, cs = h.tsqr_r(torch.from_numpy(Y).cuda(), prec="fp32")
    h.sync()
    check(oracle, Y, R, cs)
    for bad in (-1e-3, -np.inf, np.nan):
        Y = X.copy()
        Y[54_321, 6] = bad
        h.tsqr_r(torch.from_numpy(Y).cuda(), prec="fp32")
        with pytest.raises(mrnmf.MrnmfError) as e:
            h.sync()
        assert e.value.status == mrnmf.ERR_BAD_INPUT
    h.tsqr_r(torch.from_numpy(X).cuda(), prec="fp32")
    h.sync()


@pytest.mark.parametrize("n", [6, 12, 16, 24, 28])
def test_ill_conditioned_columns(h, oracle, n):
    X, _ = synth.planted_separable(400_000, n, max(2, n // 3), seed=1404000 + n, noise=1e-3, decades=6.0)
    R, cs = h.tsqr_r(torch.from_numpy(X).cuda(), prec="fp32")
    h.sync()
    Ro = oracle.qr_r(X.astype(np.float64))
    Rg = host(R)
    assert rel_fro(Rg, Ro) <= R_TOL_FP32
    col = np.linalg.norm(Rg - Ro, axis=0) / np.linalg.norm(Ro, axis=0)
    assert np.max(col) < COL_TOL_ILLCOND
