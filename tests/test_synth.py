"""Input generators (no GPU): the Kronecker workload against numpy's kron, and
the planted structure of A kron A."""
import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

torch = pytest.importorskip("torch")


def test_kron_rows_is_kron():
    A, K = synth.kron_factor(rows=200)
    At = torch.from_numpy(A)
    full = np.kron(A, A)
    assert np.array_equal(synth.kron_rows(At, 0, 200 * 200).numpy(), full)
    assert np.array_equal(synth.kron_rows(At, 12345, 999).numpy(), full[12345:12345 + 999])


def test_kron_planted_columns_generate_the_rest():
    # noise-free factor: A = A(:,K_A) H_A, so A kron A = (A kron A)(:, K) (H_A kron H_A)
    w = synth.Workload("t", 0, 25, 16, 32, seed=77)
    A, K = synth.kron_factor(w, rows=300)
    X = np.kron(A, A)
    H, res, rank, _ = np.linalg.lstsq(X[:, K], X, rcond=None)
    assert rank == 16
    assert np.linalg.norm(X[:, K] @ H - X) <= 1e-10 * np.linalg.norm(X)
    assert len(K) == 16 and len(set(K.tolist())) == 16


def test_planted_structure_is_separable():
    # X = W [I H'] Pi (Sec. 4's generator): X(:,K) H_true = X exactly without
    # noise, the columns of H' lie in the simplex, and the scaling moves with
    # the permutation
    X, P = synth.planted_separable(3000, 20, 6, seed=5, dtype=np.float64, decades=3.0)
    assert len(P.K) == 6 and np.all(np.diff(P.K) > 0)
    np.testing.assert_allclose(X[:, P.K] @ P.H_true, X, rtol=1e-12, atol=1e-12)
    Hp = P.Hmix / P.colscale[None, :]
    others = np.setdiff1d(np.arange(20), P.K)
    np.testing.assert_allclose(Hp[:, others].sum(0), 1.0, rtol=1e-12)
    assert np.all(Hp >= 0)
    assert np.all((P.colscale >= 1.0) & (P.colscale <= 1e3))


def test_whole_chunks_regenerate_alone():
    # chunk c is drawn from (seed, c) alone: the whole chunks of a longer X are
    # those of a shorter one, and a chunk can be regenerated by itself
    X, P = synth.planted_separable(3 * synth.CHUNK_ROWS // 2, 10, 4, seed=9, noise=1e-3)
    Xs, _ = synth.planted_separable(synth.CHUNK_ROWS + 100, 10, 4, seed=9, noise=1e-3)
    assert np.array_equal(X[:synth.CHUNK_ROWS], Xs[:synth.CHUNK_ROWS])
    c1 = synth.rows_chunk(P, 9, 1, synth.CHUNK_ROWS // 2, noise=1e-3)
    assert np.array_equal(c1, X[synth.CHUNK_ROWS:])
    assert np.all(X >= 0)


def test_batch_shapes_follow_their_recipe():
    probs = synth.batch_problems(256, seed=3)
    m = np.array([p[0] for p in probs])
    n = np.array([p[1] for p in probs])
    r = np.array([p[2] for p in probs])
    assert np.all((m >= 1e4 - 1) & (m <= 1e7 + 1)) and np.all((n >= 10) & (n <= 128))
    assert np.all((r >= 3) & (r <= np.maximum(3, np.minimum(16, n // 2))))
    # log-uniform m: the median is near the geometric mean of the range
    assert 1e5 < np.median(m) < 1e6
