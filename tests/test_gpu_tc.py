"""The tcgen05 datapath (mrnmf_tc_selftest): D = A B^T on the tensor cores
against a float64 host GEMM, for the three input forms.  Bounds are the
forms' elementwise rounding bounds times |A| |B|^T."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrnmf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_6964_gb300 import build, mrnmf as m
    build.build()
    return m


@pytest.mark.parametrize("kind,bound", [("tf32", 2.0 ** -9), ("tf32x3", 2.0 ** -19), ("bf16", 2.0 ** -6)])
@pytest.mark.parametrize("N,K", [(16, 32), (64, 64), (128, 64), (256, 32)])
def test_tc_gemm(mrnmf, kind, bound, N, K):
    g = np.random.default_rng(N * 1000 + K)
    A = g.standard_normal((128, K)).astype(np.float32)
    B = g.standard_normal((N, K)).astype(np.float32)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    D = mrnmf.tc_selftest(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), kind, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    err = np.abs(D.cpu().numpy() - ref)
    assert np.all(err <= bound * scale + 1e-6), float(np.max(err / scale))


def test_tc_projection_pass_matches_oracle():
    """The tcgen05 (3-pass TF32) projection pass, selected with MRNMF_GP_TC=1,
    against the oracle's G^T X within the same bound as the SIMT pass."""
    import os
    import subprocess
    import sys
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    code = r"""
import sys, numpy as np, torch
sys.path.insert(0, '.')
import oracle
from paper_1402_6964_gb300 import mrnmf, synth
for m, n, k in [(1000, 7, 3), (40013, 50, 20), (9001, 128, 64)]:
    X = synth.random_nonneg(m, n, seed=m + n)
    h = mrnmf.Handle()
    GX, cs = h.gauss_project(torch.from_numpy(X).cuda(), k, seed=77, row_offset=5)
    h.sync()
    X64 = X.astype(np.float64)
    GXo = oracle.gauss_project(X64, k, 77, row0=5)
    G = oracle.gauss_matrix(77, 5, m, k)
    bound = 2e-6 * (np.abs(G).T @ np.abs(X64)) + 1e-12
    assert np.all(np.abs(GX.cpu().numpy() - GXo) <= bound), (m, n, k)
    np.testing.assert_allclose(cs.cpu().numpy(), oracle.colsum(X64), rtol=1e-6)
print("ok")
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, MRNMF_GP_TC="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
