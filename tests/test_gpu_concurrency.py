"""The n-by-n step run the way the benchmark runs it: the SPA, XRAY and GP
chains (selection, NNLS, residual) on three CUDA streams with one handle each,
eagerly and replayed from a captured CUDA graph.

Every chain reads only R, the column sums and GX, so the concurrent and the
graph-replayed forms must give bit for bit what the sequential calls give on
one handle, and K must equal the FP64 oracle's on the same input (the input
here is the oracle's own R, so the picks are not tie-ambiguous).  The graph is
replayed after R changes, to check that it reads the current buffers.
"""
import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

METHODS = ("xray", "spa", "gp")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_6964_gb300 import build, mrnmf
    build.build()
    return mrnmf


def problem(oracle, seed, n=40, r=8, k=16):
    X, P = synth.planted_separable(30000, n, r, seed=seed, noise=1e-3)
    X64 = X.astype(np.float64)
    return oracle.qr_r(X64), oracle.colsum(X64), oracle.gauss_project(X64, k, 11), r


class Chains:
    """Fixed device buffers and one handle and stream per method."""

    def __init__(self, lib, n, r, k):
        d = "cuda"
        self.R = torch.zeros((n, n), dtype=torch.float64, device=d)
        self.cs = torch.zeros(n, dtype=torch.float64, device=d)
        self.GX = torch.zeros((k, n), dtype=torch.float64, device=d)
        self.K = {m: (torch.empty(r, dtype=torch.int32, device=d), torch.empty(r, dtype=torch.float64, device=d))
                  for m in METHODS}
        self.H = {m: torch.empty((r, n), dtype=torch.float64, device=d) for m in METHODS}
        self.out = {m: torch.empty(2, dtype=torch.float64, device=d) for m in METHODS}
        self.side = {m: (torch.cuda.Stream(), lib.Handle()) for m in METHODS}
        self.ev0 = torch.cuda.Event()
        self.ev = {m: torch.cuda.Event() for m in METHODS}
        self.r = r

    def load(self, R, cs, GX):
        self.R.copy_(torch.from_numpy(R))
        self.cs.copy_(torch.from_numpy(cs))
        self.GX.copy_(torch.from_numpy(GX))

    def run(self, main):
        self.ev0.record(main)
        for m in METHODS:
            s, hm = self.side[m]
            s.wait_event(self.ev0)
            hm.select_extreme(m, R=self.R, colsum=self.cs, GX=self.GX if m == "gp" else None, r=self.r,
                              out=self.K[m], stream=s)
            hm.nnls_h(self.R, self.K[m][0], out=self.H[m], stream=s)
            hm.residual(self.R, self.K[m][0], self.H[m], out=self.out[m], stream=s)
            self.ev[m].record(s)
        for m in METHODS:
            main.wait_event(self.ev[m])

    def results(self):
        torch.cuda.synchronize()
        for _, hm in self.side.values():
            hm.sync()
        return {m: (self.K[m][0].cpu().numpy().copy(), self.H[m].cpu().numpy().copy(),
                    self.out[m].cpu().numpy().copy()) for m in METHODS}

    def close(self):
        for _, hm in self.side.values():
            hm.close()


def sequential(lib, R, cs, GX, r):
    out = {}
    with lib.Handle() as h:
        Rd, csd, GXd = (torch.from_numpy(a).cuda() for a in (R, cs, GX))
        for m in METHODS:
            K, _ = h.select_extreme(m, R=Rd, colsum=csd, GX=GXd if m == "gp" else None, r=r)
            H = h.nnls_h(Rd, K)
            o = h.residual(Rd, K, H)
            h.sync()
            out[m] = (K.cpu().numpy(), H.cpu().numpy(), o.cpu().numpy())
    return out


def check_against(got, want, oracle, R, cs, GX, r):
    for m in METHODS:
        np.testing.assert_array_equal(got[m][0], want[m][0])
        np.testing.assert_array_equal(got[m][1], want[m][1])
        np.testing.assert_array_equal(got[m][2], want[m][2])
    assert list(got["spa"][0]) == list(oracle.spa(R, cs, r)[0])
    assert list(got["xray"][0]) == list(oracle.xray(R, r)[0])
    assert list(got["gp"][0]) == list(oracle.gp_select(GX, cs, r)[0])


def test_three_streams_match_sequential(lib, oracle):
    R, cs, GX, r = problem(oracle, 31)
    c = Chains(lib, R.shape[0], r, GX.shape[0])
    try:
        c.load(R, cs, GX)
        main = torch.cuda.current_stream()
        for _ in range(3):
            c.run(main)
        check_against(c.results(), sequential(lib, R, cs, GX, r), oracle, R, cs, GX, r)
    finally:
        c.close()


def test_graph_replay_matches_and_follows_inputs(lib, oracle):
    R1, cs1, GX1, r = problem(oracle, 32)
    R2, cs2, GX2, _ = problem(oracle, 33)
    c = Chains(lib, R1.shape[0], r, GX1.shape[0])
    try:
        main = torch.cuda.current_stream()
        c.load(R1, cs1, GX1)
        c.run(main)  # warm-up: every workspace is allocated here
        c.results()
        cap = torch.cuda.Stream()
        cap.wait_stream(main)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            c.run(cap)
        main.wait_stream(cap)
        torch.cuda.synchronize()
        for R, cs, GX in ((R2, cs2, GX2), (R1, cs1, GX1)):
            c.load(R, cs, GX)
            g.replay()
            check_against(c.results(), sequential(lib, R, cs, GX, r), oracle, R, cs, GX, r)
    finally:
        c.close()
