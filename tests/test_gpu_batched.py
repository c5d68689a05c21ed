"""Batched pass (mrnmf_tsqr_r_batched) against the oracle, problem by
problem: uneven m (1 .. 1e5 rows) and n (1 .. 128, all three kernel
families), and the same batch captured in a CUDA graph and replayed."""
import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R_TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_6964_gb300 import build, mrnmf
    build.build()
    hd = mrnmf.Handle()
    yield hd
    hd.close()


def _batch(seed, count):
    g = np.random.default_rng(seed)
    shapes = [(1, 1), (64, 64), (129, 33), (5000, 20), (77777, 50), (3000, 100), (100000, 7), (20011, 128)]
    while len(shapes) < count:
        n = int(g.integers(1, 129))
        m = int(max(n, round(np.exp(g.uniform(np.log(max(n, 10)), np.log(60000))))))
        shapes.append((m, n))
    return [synth.random_nonneg(m, n, seed=seed + 17 * i) for i, (m, n) in enumerate(shapes)]


def _check(oracle, Xs, outs):
    for X, (R, cs) in zip(Xs, outs):
        X64 = X.astype(np.float64)
        Ro = oracle.qr_r(X64)
        Rg = R.cpu().numpy()
        assert np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro) <= R_TOL_FP32, X.shape
        np.testing.assert_allclose(cs.cpu().numpy(), oracle.colsum(X64), rtol=1e-6)


def test_batched_matches_oracle(h, oracle):
    Xs = _batch(5, 24)
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    outs = h.tsqr_r_batched(Xd)
    h.sync()
    _check(oracle, Xs, outs)


def test_batched_graph_replay(h, oracle):
    Xs = _batch(9, 12)
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    outs = h.tsqr_r_batched(Xd)  # sizes the handle's buffers
    h.sync()
    for R, cs in outs:
        R.zero_()
        cs.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            h.tsqr_r_batched(Xd, outs=outs, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    h.sync()
    _check(oracle, Xs, outs)


def test_batched_select_nnls_residual_matches_oracle(h, oracle):
    """The separable step on each batched R, for the problems of a drawn batch
    of the 256-problem workload's distribution (m log-uniform in [1e4, 1e7],
    n in 10..128, r in 3..min(16, n/2), sigma = 1e-3) whose m is at most
    2e5 (the oracle's QR of the larger members takes minutes): SPA's and
    XRAY's K under the margin rule (SPA also = the planted K), and H and the
    residual within relative 1e-4 wherever K matches."""
    from test_gpu_parity import compare_K, k_margin
    probs = [p for p in synth.batch_problems(40, seed=1402005) if p[0] <= 200_000]
    assert len(probs) >= 8
    data = [synth.planted_separable(m, n, r, seed=1402005 + 31 * i, noise=1e-3) for i, (m, n, r) in enumerate(probs)]
    Xd = [torch.from_numpy(X).cuda() for X, _ in data]
    outs = h.tsqr_r_batched(Xd)
    h.sync()
    for (m, n, r), (X, P), (R, cs) in zip(probs, data, outs):
        X64 = X.astype(np.float64)
        Ro, so = oracle.qr_r(X64), oracle.colsum(X64)
        Rg = R.cpu().numpy()
        assert np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro) <= R_TOL_FP32, (m, n)
        for method in ("spa", "xray"):
            K, gap = h.select_extreme(method, R=R, colsum=cs, r=r)
            H = h.nnls_h(R, K)
            out = h.residual(R, K, H)
            h.sync()
            Kg = K.cpu().numpy()
            if method == "spa":
                Ko, go = oracle.spa(Ro, so, r)
            else:
                Ko, go, _ = oracle.xray(Ro, r)
            t = compare_K(Kg, Ko, go, k_margin(Rg, Ro), n=n)
            if t == r:
                Ho, _ = oracle.nnls_h(Ro, Ko)
                Hg = H.cpu().numpy()
                assert np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho) <= 1e-4, (m, n, r, method)
                ab, rel = oracle.residual(Ro, Ko, Ho)
                assert out.cpu().numpy()[0] == pytest.approx(ab, rel=1e-4)
            if method == "spa":
                assert sorted(Kg) == list(P.K), (m, n, r)
