"""The pass at the benchmarked full sizes, checked through properties that hold
at any size (the oracle cannot run these), plus empty stream chunks.

  1e8 x 200 ill-conditioned (80 GB, drawn on the device), k = 40:
    R'R = X'X (binary64 Gram accumulated on the device): relative 2e-5
    column sums = binary64 sums of X: relative 1e-6
    GX of the fused pass = GX of the projection-only pass (a different kernel): relative 1e-5
    SPA on R recovers the planted K (Sec. 4)
  1.6e9 x 25 flow-cytometry-shaped stream (24 chunks of 64M rows, k = 16):
    R'R = X'X over all chunks, column sums, SPA recovers the planted K
"""
import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROWS_G = 1 << 20  # Gram accumulation chunk


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


def gram_and_sums(X, G=None, s=None):
    n = X.shape[1]
    if G is None:
        G = torch.zeros((n, n), dtype=torch.float64, device=X.device)
        s = torch.zeros(n, dtype=torch.float64, device=X.device)
    for c0 in range(0, X.shape[0], ROWS_G):
        Xc = X[c0:c0 + ROWS_G].double()
        G += Xc.T @ Xc
        s += Xc.sum(0)
        del Xc
    return G, s


def test_full_size_ill_conditioned_1e8x200(h):
    w = synth.WORKLOADS["illcond_1e8x200"]
    P = synth.planted_structure(w.n, w.r, w.seed, w.alpha, w.decades)
    X = torch.empty((w.m, w.n), dtype=torch.float32, device="cuda")
    ch = 1 << 23
    for c0 in range(0, w.m, ch):
        rows = min(ch, w.m - c0)
        synth.device_planted(rows, w.n, w.r, w.seed, noise=w.noise, alpha=w.alpha, w_dist=w.w_dist,
                             chunk=c0 // ch, P=P, out=X[c0:c0 + rows])
    R, cs, GX = h.tsqr_gp(X, w.k, w.seed)
    K, gap = h.select_extreme("spa", R=R, colsum=cs, r=w.r)
    GX2, cs2 = h.gauss_project(X, w.k, w.seed, row_offset=0)
    h.sync()
    G, s = gram_and_sums(X)
    del X
    Rg = host(R)
    Gh = host(G)
    assert np.linalg.norm(Rg.T @ Rg - Gh) <= 2e-5 * np.linalg.norm(Gh)
    np.testing.assert_allclose(host(cs), host(s), rtol=1e-6)
    np.testing.assert_allclose(host(cs2), host(s), rtol=1e-6)
    assert np.linalg.norm(host(GX) - host(GX2)) <= 1e-5 * np.linalg.norm(host(GX2))
    assert sorted(host(K).tolist()) == P.K.tolist()


def test_full_size_stream_1p6e9x25(h):
    w = synth.WORKLOADS["fc_stream_1p6e9x25"]
    P = synth.planted_structure(w.n, w.r, w.seed, w.alpha)
    chunk = 64 << 20
    buf = torch.empty((chunk, w.n), dtype=torch.float32, device="cuda")
    h.stream_begin(w.n, k=w.k, seed=w.seed)
    G = s = None
    for c in range((w.m + chunk - 1) // chunk):
        rows = min(chunk, w.m - c * chunk)
        X, _ = synth.device_planted(rows, w.n, w.r, w.seed, noise=w.noise, alpha=w.alpha, w_dist=w.w_dist,
                                    chunk=c, P=P, out=buf[:rows])
        h.stream_push(X)
        G, s = gram_and_sums(X, G, s)  # same stream: the next chunk overwrites buf only afterwards
    R, cs, GX = h.stream_end(w.n, k=w.k)
    K, gap = h.select_extreme("spa", R=R, colsum=cs, r=w.r)
    h.sync()
    Rg = host(R)
    Gh = host(G)
    assert np.linalg.norm(Rg.T @ Rg - Gh) <= 2e-5 * np.linalg.norm(Gh)
    np.testing.assert_allclose(host(cs), host(s), rtol=1e-6)
    assert sorted(host(K).tolist()) == P.K.tolist()


def test_stream_with_empty_chunks(h, oracle):
    X = synth.random_nonneg(20000, 40, seed=23)
    Xd = torch.from_numpy(X).cuda()
    h.stream_begin(40, k=4, seed=5)
    for a, b in [(0, 0), (0, 7000), (7000, 7000), (7000, 20000), (20000, 20000)]:
        h.stream_push(Xd[a:b])
    R, cs, GX = h.stream_end(40, k=4)
    h.sync()
    X64 = X.astype(np.float64)
    Ro = oracle.qr_r(X64)
    assert np.linalg.norm(host(R) - Ro) <= 1e-5 * np.linalg.norm(Ro)
    np.testing.assert_allclose(host(cs), oracle.colsum(X64), rtol=1e-6)
