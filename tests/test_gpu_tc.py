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
