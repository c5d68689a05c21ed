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


def _bf16(a):
    """Round binary32 values to bfloat16, to nearest with ties to even, on the
    bit pattern (finite inputs): add 0x7fff plus the lowest kept bit, truncate."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _bf16_ambiguity(G, rel):
    """Per entry of binary32 G, the gap between its two bfloat16 neighbours
    where G lies within rel |G| of their midpoint (else 0).  The device draws G
    with its own log, sqrt and sin/cos, equal to the oracle's to a few binary32
    ulps, so such an entry may round to either neighbour there."""
    g = np.ascontiguousarray(G, dtype=np.float32)
    u = g.view(np.uint32)
    lo = (u & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    hi = ((u & np.uint32(0xFFFF0000)) + np.uint32(0x10000)).view(np.float32).astype(np.float64)
    mid = 0.5 * (lo + hi)
    g64 = g.astype(np.float64)
    return np.where(np.abs(g64 - mid) <= rel * np.abs(g64), np.abs(hi - lo), 0.0)


def test_bf16_rounding_helper():
    # 1 + 2^-8 (exactly half an ulp of bfloat16 at 1) ties to even: 1; 1 + 3 * 2^-8 ties up to 1 + 2^-6
    v = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -2.5, 0.0], dtype=np.float32)
    assert _bf16(v).tolist() == [1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -2.5, 0.0]
    amb = _bf16_ambiguity(np.array([1 + 2 ** -8, 1.0, -(1 + 2 ** -8)], dtype=np.float32), 8 * 2.0 ** -24)
    assert amb.tolist() == [2 ** -7, 0.0, 2 ** -7]


@pytest.mark.parametrize("m,n,k,row0", [(33, 1, 1, 0), (1000, 7, 3, 5), (40013, 50, 20, 0), (9001, 128, 64, 123_456_789)])
def test_bf16_projection_matches_oracle_on_rounded_inputs(m, n, k, row0):
    """mrnmf_gauss_project_tc, form BF16: G'X equals the FP64 product of the
    oracle's G and of X, both rounded to bfloat16, within the binary32
    accumulation bound 2e-6 |G|'|X| elementwise, plus, for the entries of G
    within 8 binary32 ulps of a bfloat16 rounding midpoint (either rounding is
    then valid), their rounding gap times |X|; and it is that product, not the
    unrounded one (the rounding moves some entries far past the bound)."""
    import oracle as orc
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_6964_gb300 import build, mrnmf, synth
    build.build()
    X = synth.random_nonneg(m, n, seed=m + 3 * n)
    h = mrnmf.Handle()
    GX, cs = h.gauss_project_tc(torch.from_numpy(X).cuda(), k, seed=91, form="bf16", row_offset=row0)
    h.sync()
    h.close()
    G = orc.gauss_matrix(91, row0, m, k)
    Gb, Xb = _bf16(G).astype(np.float64), _bf16(X).astype(np.float64)
    ref = Gb.T @ Xb
    amb = _bf16_ambiguity(G, 8 * 2.0 ** -24)
    bound = 2e-6 * (np.abs(Gb).T @ np.abs(Xb)) + amb.T @ np.abs(Xb) + 1e-12
    got = GX.cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))
    np.testing.assert_allclose(cs.cpu().numpy(), orc.colsum(X.astype(np.float64)), rtol=1e-6)
    if m >= 1000:
        full = G.T @ X.astype(np.float64)
        assert np.max(np.abs(got - full) / bound) > 10.0


def test_tf32x3_projection_by_name_matches_oracle():
    """The same entry point with form TF32X3 (no environment variable): the
    oracle's G'X within the SIMT pass's bound."""
    import oracle as orc
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_6964_gb300 import build, mrnmf, synth
    build.build()
    h = mrnmf.Handle()
    for m, n, k in [(1000, 7, 3), (40013, 50, 20), (9001, 128, 64)]:
        X = synth.random_nonneg(m, n, seed=m + n)
        GX, cs = h.gauss_project_tc(torch.from_numpy(X).cuda(), k, seed=77, form="tf32x3", row_offset=5)
        h.sync()
        X64 = X.astype(np.float64)
        G = orc.gauss_matrix(77, 5, m, k)
        bound = 2e-6 * (np.abs(G).T @ np.abs(X64)) + 1e-12
        assert np.all(np.abs(GX.cpu().numpy() - orc.gauss_project(X64, k, 77, row0=5)) <= bound), (m, n, k)
        np.testing.assert_allclose(cs.cpu().numpy(), orc.colsum(X64), rtol=1e-6)
    h.close()


def _agree_under_margin(Kg, Ko, gap, margin, n):
    """Picks agree at every step whose oracle gap exceeds `margin`; from the
    first divergence at a smaller gap on, only validity is checked (distinct
    indices in [0, n))."""
    Kg = [int(v) for v in Kg]
    assert len(set(Kg)) == len(Kg) and all(0 <= v < n for v in Kg), Kg
    for t in range(len(Ko)):
        if Kg[t] != Ko[t]:
            assert gap[t] < margin, (t, Kg[t], Ko[t], gap[t], margin)
            return t
    return len(Ko)


def test_gp_selection_on_bf16_projection_matches_oracle():
    """GP selection (Sec. 2.3) on the BF16 projection: K against the oracle's GP
    run on the bfloat16-rounded G and X with binary64 sums, and against the
    oracle's GP on the unrounded inputs, each under the margin rule (100 times
    the relative error of that comparison's GX); both recover the planted
    columns of the near-separable input."""
    import oracle as orc
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_6964_gb300 import build, mrnmf, synth
    build.build()
    m, n, r, k, seed = 200_000, 50, 10, 20, 7
    X, P = synth.planted_separable(m, n, r, seed=1402002, noise=1e-3)
    X64 = X.astype(np.float64)
    h = mrnmf.Handle()
    GX, cs = h.gauss_project_tc(torch.from_numpy(X).cuda(), k, seed=seed, form="bf16")
    K, gap = h.select_extreme("gp", colsum=cs, GX=GX, r=r)
    h.sync()
    h.close()
    got, Kg = GX.cpu().numpy(), K.cpu().numpy()
    G = orc.gauss_matrix(seed, 0, m, k)
    so = orc.colsum(X64)
    for ref in (_bf16(G).astype(np.float64).T @ _bf16(X).astype(np.float64), G.T @ X64):
        Ko, _, go = orc.gp_select(ref, so, r)
        margin = max(100.0 * float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))), 1e-12)
        _agree_under_margin(Kg, Ko, go, margin, n)
    assert sorted(int(v) for v in Kg) == list(P.K)
