"""The projection-only pass on the SIMT warp kernel (n <= 64, k <= 32) against
the FP64 oracle.

GX is checked entry by entry against the oracle's G'X within 2e-6 of
|G|'|X| (binary32 products and sums over at most 32 rows a tile, binary64
across tiles); the column sums within relative 1e-6.  Cases:

* widths on both sides of one and two columns a lane (1, 7, 25, 32, 33, 50, 64)
  and k from 1 to 32, k not a multiple of 4 included;
* row counts below one tile, ragged, and large enough that every stream
  flushes its binary32 partials to binary64 several times;
* strided rows and a base off the 16-byte grid (the direct-load path);
* a row offset (the Gaussian key of row 0), as a stream's later chunks use;
* the input check: a negative entry or NaN is reported, -0 passes.
"""
import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GX_TOL = 2e-6
CS_RTOL = 1e-6


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_6964_gb300 import build, mrnmf
    build.build()
    hd = mrnmf.Handle()
    yield hd
    hd.close()


def host(t):
    return t.detach().cpu().numpy()


def gx_bound(X, k, seed, row0=0):
    import oracle as orc
    G = orc.gauss_matrix(seed, row0, X.shape[0], k)
    return np.abs(G).T @ np.abs(X.astype(np.float64))


def check_gx(oracle, X, k, seed, GX, cs=None, row0=0):
    X64 = X.astype(np.float64)
    GXo = oracle.gauss_project(X64, k, seed, row0=row0)
    err = np.abs(host(GX) - GXo)
    assert np.all(err <= GX_TOL * gx_bound(X, k, seed, row0) + 1e-12), float(err.max())
    if cs is not None:
        np.testing.assert_allclose(host(cs), oracle.colsum(X64), rtol=CS_RTOL)


@pytest.mark.parametrize("n,k", [(1, 1), (7, 3), (25, 16), (32, 32), (33, 5), (50, 20), (64, 32), (64, 1)])
def test_widths_and_k(h, oracle, n, k):
    for m in (n, 31, 4099, 100_003):
        if m < n:
            continue
        X = synth.random_nonneg(m, n, seed=7 * n + k + m)
        GX, cs = h.gauss_project(torch.from_numpy(X).cuda(), k, seed=1234 + n, row_offset=0)
        h.sync()
        check_gx(oracle, X, k, 1234 + n, GX, cs)


@pytest.mark.parametrize("m,n,k", [(3_000_017, 8, 12), (2_600_000, 50, 20)])
def test_many_tiles_per_stream(h, oracle, m, n, k):
    # more than 32 tiles a stream: the binary32 partials are flushed several times
    X = synth.random_nonneg(m, n, seed=m % 977 + n)
    GX, cs = h.gauss_project(torch.from_numpy(X).cuda(), k, seed=5, row_offset=0)
    h.sync()
    check_gx(oracle, X, k, 5, GX, cs)


@pytest.mark.parametrize("n", [9, 40])
def test_direct_load_paths(h, oracle, n):
    W = synth.random_nonneg(20_001, n + 3, seed=n)
    Xs = torch.from_numpy(W).cuda()[:, 1:1 + n]              # ldx = n + 3
    GX, cs = h.gauss_project(Xs, 10, seed=8, row_offset=0)
    h.sync()
    check_gx(oracle, np.ascontiguousarray(W[:, 1:1 + n]), 10, 8, GX, cs)
    flat = torch.from_numpy(synth.random_nonneg(20_001 * n + 1, 1, seed=n + 1).ravel()).cuda()
    Xo = flat[1:].view(20_001, n)                            # base 4 bytes off the 16-byte grid
    assert Xo.data_ptr() % 16 != 0
    GX, cs = h.gauss_project(Xo, 10, seed=8, row_offset=0)
    h.sync()
    check_gx(oracle, host(Xo), 10, 8, GX, cs)


def test_row_offset(h, oracle):
    X = synth.random_nonneg(50_000, 50, seed=3)
    GX, _ = h.gauss_project(torch.from_numpy(X).cuda(), 20, seed=11, row_offset=7_000_000_123)
    h.sync()
    check_gx(oracle, X, 20, 11, GX, row0=7_000_000_123)


def test_input_check(h):
    from paper_1402_6964_gb300 import mrnmf
    X = synth.random_nonneg(60_000, 50, seed=4)
    Y = X.copy()
    Y[::501, 7] = -0.0
    h.gauss_project(torch.from_numpy(Y).cuda(), 20, seed=1, row_offset=0)
    h.sync()
    for bad in (-1e-3, np.nan):
        Y = X.copy()
        Y[40_001, 45] = bad
        h.gauss_project(torch.from_numpy(Y).cuda(), 20, seed=1, row_offset=0)
        with pytest.raises(mrnmf.MrnmfError) as e:
            h.sync()
        assert e.value.status == mrnmf.ERR_BAD_INPUT
