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
