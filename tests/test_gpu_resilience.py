"""Checkpoint and resume of a stream, and the bounded device waits, through the C ABI.

Checkpoint/resume (the device analogue of re-running a failed map task,
Sec. 3.5): a stream interrupted after some chunks, its state saved to host,
the handle destroyed, the state loaded into a fresh handle and the remaining
chunks pushed, must give R, the column sums and GX bit for bit equal to the
uninterrupted stream -- and both within the usual bounds of the oracle.

Bounded waits: a missing mbarrier arrival in the leaf's hand-over must end in
MRNMF_ERR_TIMEOUT on the status word, with the later waits abandoned, and the
context must stay usable afterwards.  No fault, trap or hang is involved.
"""
import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_6964_gb300 import build, mrnmf
    build.build()
    return mrnmf


def host(t):
    return t.detach().cpu().numpy()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# warp leaf with and without GX, the wide-tree boundary, the pipelined leaf,
# binary64 input, the tensor-core form
CASES = [
    (60000, 50, 16, "f32", "auto"),
    (45000, 25, 0, "f32", "auto"),
    (30000, 128, 8, "f32", "auto"),
    (20000, 200, 20, "f32", "auto"),
    (25000, 40, 8, "f64", "auto"),
    (30000, 36, 8, "f32", "tf32x3"),
]
CUTS = [0, 7001, 7001, 19999, 33333]  # chunk boundaries (an empty chunk, ragged sizes)


def chunks(m):
    b = [c for c in CUTS if c < m] + [m]
    return list(zip(b[:-1], b[1:]))


@pytest.mark.parametrize("m,n,k,dt,prec", CASES)
def test_resume_is_bit_exact(lib, oracle, m, n, k, dt, prec):
    X = synth.random_nonneg(m, n, seed=1000 + n + k)
    if dt == "f64":
        X = X.astype(np.float64)
    Xd = dev(X)
    parts = chunks(m)
    seed = 77 + n

    with lib.Handle() as h:
        h.stream_begin(n, dtype=dt, prec=prec, k=k, seed=seed)
        for a, b in parts:
            h.stream_push(Xd[a:b])
        R0, cs0, GX0 = h.stream_end(n, k=k)
        h.sync()

    cut = 3  # interrupted after three chunks (one of them empty)
    h1 = lib.Handle()
    h1.stream_begin(n, dtype=dt, prec=prec, k=k, seed=seed)
    for a, b in parts[:cut]:
        h1.stream_push(Xd[a:b])
    state = h1.stream_state_save()
    h1.close()  # the process's work on the stream is lost here

    with lib.Handle() as h2:
        h2.stream_begin(n, dtype=dt, prec=prec, k=k, seed=seed)
        h2.stream_state_load(state)
        for a, b in parts[cut:]:
            h2.stream_push(Xd[a:b])
        R1, cs1, GX1 = h2.stream_end(n, k=k)
        h2.sync()

    assert torch.equal(R0, R1)
    assert torch.equal(cs0, cs1)
    if k:
        assert torch.equal(GX0, GX1)
    X64 = X.astype(np.float64)
    assert rel_fro(host(R1), oracle.qr_r(X64)) <= (1e-12 if dt == "f64" else 1e-5)
    np.testing.assert_allclose(host(cs1), oracle.colsum(X64), rtol=1e-6)


def test_state_is_checked_on_load(lib):
    X = dev(synth.random_nonneg(5000, 30, seed=3))
    with lib.Handle() as h:
        h.stream_begin(30, k=4, seed=9)
        h.stream_push(X)
        state = h.stream_state_save()
        for n, k, seed, dt in [(31, 4, 9, "f32"), (30, 5, 9, "f32"), (30, 4, 10, "f32"), (30, 4, 9, "f64")]:
            h.stream_begin(n, dtype=dt, k=k, seed=seed)
            with pytest.raises(lib.MrnmfError) as e:
                h.stream_state_load(state)
            assert e.value.status == lib.ERR_INVALID_ARG
        h.stream_begin(30, k=4, seed=9)
        bad = bytearray(state)
        bad[0] ^= 0xFF
        with pytest.raises(lib.MrnmfError) as e:
            h.stream_state_load(bytes(bad))
        assert e.value.status == lib.ERR_INVALID_ARG
        with pytest.raises(lib.MrnmfError) as e:
            h.stream_state_load(state[:-8])
        assert e.value.status == lib.ERR_INVALID_ARG
        # the handle is still good: load the real state and finish
        h.stream_state_load(state)
        h.stream_push(X)
        R, cs, _ = h.stream_end(30, k=4)
        h.sync()
        X64 = np.concatenate([host(X), host(X)]).astype(np.float64)
        np.testing.assert_allclose(host(cs), X64.sum(0), rtol=1e-6)


@pytest.mark.parametrize("missing,expect", [(0, [0, 0, 0, 0]), (1, [0, 1, 2, 2]), (2, [0, 0, 1, 2]),
                                            (3, [0, 0, 0, 1])])
def test_missing_arrival_times_out(lib, oracle, missing, expect):
    limit = 5_000_000  # 5 ms
    lib.wait_selftest(0, limit)  # module loaded before the timed call
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    out, status = lib.wait_selftest(missing, limit)
    t1.record()
    torch.cuda.synchronize()
    assert host(out).tolist() == expect
    assert int(status.item()) == (lib.ERR_TIMEOUT if missing else 0)
    if missing:
        # the wait that ran out took its limit; the abandoned ones added nothing
        ms = t0.elapsed_time(t1)
        assert missing * limit * 1e-6 * 0.9 <= ms <= (missing + 1) * limit * 1e-6
    # the context is still usable
    X = synth.random_nonneg(3000, 20, seed=missing)
    with lib.Handle() as h:
        R, cs = h.tsqr_r(dev(X))
        h.sync()
    assert rel_fro(host(R), oracle.qr_r(X.astype(np.float64))) <= 1e-5


def test_householder_scalars_match_ieee(lib):
    # the leaves' beta, d, 1/beta, 1/d (hardware approximations refined by one
    # Newton step) against the IEEE square root and reciprocals: within one
    # ulp everywhere, and equal for nearly all arguments
    g = torch.Generator().manual_seed(5)
    n = 1 << 20
    alpha = (torch.rand(n, generator=g) * 2 - 1) * torch.pow(10.0, torch.rand(n, generator=g) * 24 - 12)
    sigma = torch.pow(10.0, torch.rand(n, generator=g) * 30 - 15)
    alpha[:1000] = 0.0                     # a column with a zero pivot
    sigma[1000:2000] = alpha[1000:2000] ** 2 * 1e-12  # nearly annihilated columns
    alpha, sigma = alpha.float().cuda(), sigma.float().cuda()
    out = lib.hh_scalars_selftest(alpha, sigma)
    torch.cuda.synchronize()
    o = out.cpu()
    ours, ieee = o[:, :4], o[:, 4:]
    assert torch.isfinite(ours).all()
    ulp = (ours.view(torch.int32).long() - ieee.view(torch.int32).long()).abs()
    assert int(ulp.max()) <= 1
    assert float((ulp == 0).double().mean()) >= 0.99
