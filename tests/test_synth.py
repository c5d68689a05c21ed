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
