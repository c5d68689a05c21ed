"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs; it holds none of the method's arithmetic, so
both the CUDA path's callers and the oracle's callers can use it.

The generator follows Sec. 4 of Benson, Lee, Rajwa and Gleich (arXiv
1402.6964): X = W [I_r  H'] Pi (+ N), with W m-by-r nonnegative, the columns
of H' on the simplex, and Pi a column permutation, so the planted extreme
columns K are known.  Recipe choices that the paper leaves open (or that
differ from its text on purpose) are the workload definitions below:

* W ~ U[0,1] (the paper's choice) or log-normal(0,1);
* H' columns ~ Dirichlet(alpha) (alpha = 1 or 0.5) instead of U[0,1] entries,
  so every non-extreme column lies inside the simplex hull of the extremes;
* Pi is a seeded uniform permutation instead of the paper's i <-> 10i swap;
* noise N = sigma * N(0,1), then the sum is clipped at 0 (the paper draws
  U[0, 1e-3] noise);
* optional column scaling by 10^U(0, decades) to make X ill-conditioned.

Rows are drawn in fixed chunks whose generator state depends only on
(seed, chunk index), so any chunk of a huge X can be regenerated alone.
"""
from __future__ import annotations

import dataclasses

import numpy as np

CHUNK_ROWS = 1 << 20


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    m: int
    n: int
    r: int
    k: int                 # Gaussian-projection rows (2r)
    noise: float = 0.0
    w_dist: str = "uniform"
    alpha: float = 1.0
    decades: float = 0.0
    dtype: str = "f32"
    seed: int = 0


WORKLOADS = {
    "exact_fp64": Workload("exact separable FP64, 20000x20, r=5", 20_000, 20, 5, 10,
                           dtype="f64", seed=1402001),
    "near_sep_1e7x50": Workload("near-separable FP32, 1e7x50, r=10, sigma=1e-3", 10_000_000, 50, 10, 20,
                                noise=1e-3, seed=1402002),
    "illcond_1e8x200": Workload("ill-conditioned FP32, 1e8x200, r=20, cond~1e6", 100_000_000, 200, 20, 40,
                                noise=1e-3, decades=6.0, seed=1402003),
    "fc_stream_1p6e9x25": Workload("flow-cytometry-shaped stream FP32, 1.6e9x25, r=8", 1_600_000_000, 25, 8, 16,
                                   noise=1e-2, w_dist="lognormal", alpha=0.5, seed=1402004),
    # X = A kron A with A a 40,000 x 5 near-separable factor (r_A = 4): the
    # structure of the flow-cytometry matrix of Sec. 5.2 (its data itself is
    # not available); A kron A is separable with the r_A^2 = 16 columns
    # K_A kron K_A (up to the noise in A).
    "kron_fc_1p6e9x25": Workload("Kronecker-structured stream FP32, (4e4x5) kron (4e4x5) = 1.6e9x25, r=16",
                                 1_600_000_000, 25, 16, 32, noise=1e-3, w_dist="lognormal", alpha=0.5,
                                 seed=1402005),
}

KRON_FACTOR_ROWS, KRON_FACTOR_COLS, KRON_FACTOR_RANK = 40_000, 5, 4


def _rng(*key) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(k) for k in key])))


@dataclasses.dataclass
class Planted:
    """Structure shared by every row chunk of one synthetic X."""
    n: int
    r: int
    perm: np.ndarray        # X[:, c] = (W [I H'])[:, perm[c]]
    Hmix: np.ndarray        # r-by-n, = [I H'][:, perm] * colscale
    colscale: np.ndarray    # n
    K: np.ndarray           # planted extreme columns, ascending
    H_true: np.ndarray      # r-by-n with X_noisefree = X(:,K) H_true


def planted_structure(n: int, r: int, seed: int, alpha: float = 1.0, decades: float = 0.0) -> Planted:
    if not (1 <= r <= n):
        raise ValueError("need 1 <= r <= n")
    g = _rng(seed, 0)
    Hp = g.dirichlet(np.full(r, alpha), size=n - r).T if n > r else np.zeros((r, 0))
    H0 = np.concatenate([np.eye(r), Hp], axis=1)
    perm = g.permutation(n)
    scale = 10.0 ** g.uniform(0.0, decades, size=n) if decades > 0 else np.ones(n)
    Hmix = H0[:, perm] * scale[None, :]
    K = np.sort(np.nonzero(perm < r)[0]).astype(np.int32)
    # X(:, K[t]) = W[:, perm[K[t]]] * scale[K[t]]
    q = perm[K]
    H_true = H0[q][:, perm] * (scale[None, :] / scale[K][:, None])
    return Planted(n, r, perm, Hmix, scale, K, H_true)


def rows_chunk(P: Planted, seed: int, chunk: int, rows: int, noise: float = 0.0,
               w_dist: str = "uniform", dtype=np.float32) -> np.ndarray:
    """Rows [chunk*CHUNK_ROWS, chunk*CHUNK_ROWS + rows) of X, drawn from (seed, chunk) only."""
    g = _rng(seed, 1, chunk)
    if w_dist == "uniform":
        W = g.random((rows, P.r))
    elif w_dist == "lognormal":
        W = g.lognormal(0.0, 1.0, size=(rows, P.r))
    else:
        raise ValueError(w_dist)
    X = W @ P.Hmix
    if noise > 0:
        X += noise * g.standard_normal((rows, P.n))
        np.maximum(X, 0.0, out=X)
    return X.astype(dtype, copy=False)


def planted_separable(m: int, n: int, r: int, seed: int, noise: float = 0.0, w_dist: str = "uniform",
                      alpha: float = 1.0, decades: float = 0.0, dtype=np.float32):
    """Whole X (m-by-n, row-major) plus its planted structure."""
    P = planted_structure(n, r, seed, alpha, decades)
    X = np.empty((m, n), dtype=dtype)
    for c0 in range(0, m, CHUNK_ROWS):
        rows = min(CHUNK_ROWS, m - c0)
        X[c0:c0 + rows] = rows_chunk(P, seed, c0 // CHUNK_ROWS, rows, noise, w_dist, dtype)
    return X, P


def workload_matrix(w: Workload, m: int | None = None):
    """X for a named workload (optionally truncated to its first m rows)."""
    dt = np.float64 if w.dtype == "f64" else np.float32
    return planted_separable(w.m if m is None else m, w.n, w.r, w.seed, w.noise, w.w_dist,
                             w.alpha, w.decades, dt)


def batch_problems(count: int, seed: int, m_lo: float = 1e4, m_hi: float = 1e7, n_lo: int = 10,
                   n_hi: int = 128, r_lo: int = 3, r_cap: int = 16):
    """(m, n, r) triples of a batch of independent problems: m log-uniform in
    [m_lo, m_hi], n uniform in {n_lo..n_hi}, r uniform in {r_lo..min(r_cap, n/2)}."""
    g = _rng(seed, 7)
    out = []
    for _ in range(count):
        m = int(round(np.exp(g.uniform(np.log(m_lo), np.log(m_hi)))))
        n = int(g.integers(n_lo, n_hi + 1))
        r = int(g.integers(r_lo, max(r_lo, min(r_cap, n // 2)) + 1))
        out.append((max(m, n), n, r))
    return out


def random_nonneg(m: int, n: int, seed: int, dtype=np.float32, integer: bool = False) -> np.ndarray:
    """Plain nonnegative test matrix (U[0,1), or small integers for exact-Gram checks)."""
    g = _rng(seed, 3)
    if integer:
        return g.integers(0, 8, size=(m, n)).astype(dtype)
    return g.random((m, n)).astype(dtype)


def device_planted(m: int, n: int, r: int, seed: int, noise: float = 0.0, alpha: float = 1.0, device="cuda",
                   w_dist: str = "uniform", chunk: int = 0, P: Planted | None = None, out=None):
    """The planted separable X of `planted_separable` drawn on the GPU with
    torch's counter-based generator (same recipe, different stream of random
    numbers): for workloads too large to draw on the host.  float32.  `chunk`
    selects an independent block of rows (same planted structure P)."""
    import torch
    if P is None:
        P = planted_structure(n, r, seed, alpha)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + 11 + 7919 * int(chunk))
    if w_dist == "lognormal":
        W = torch.randn((m, r), generator=g, device=device, dtype=torch.float32).exp_()
    else:
        W = torch.rand((m, r), generator=g, device=device, dtype=torch.float32)
    H = torch.from_numpy(P.Hmix.astype(np.float32)).to(device)
    X = torch.matmul(W, H, out=out) if out is not None else W @ H
    del W
    if noise > 0:
        X.add_(torch.randn((m, n), generator=g, device=device, dtype=torch.float32), alpha=noise)
        X.clamp_(min=0.0)
    return X, P


def kron_factor(w: Workload = None, rows: int = KRON_FACTOR_ROWS):
    """The factor A (rows x 5, binary64, r_A = 4) of a Kronecker workload and
    the planted K of A kron A: {p*5 + q : p, q in K_A}, ascending."""
    w = w or WORKLOADS["kron_fc_1p6e9x25"]
    A, PA = planted_separable(rows, KRON_FACTOR_COLS, KRON_FACTOR_RANK, w.seed, w.noise, w.w_dist, w.alpha,
                              dtype=np.float64)
    K = np.array(sorted(int(p) * KRON_FACTOR_COLS + int(q) for p in PA.K for q in PA.K), np.int32)
    return A, K


def kron_rows(A, start: int, count: int, out=None):
    """Rows start .. start+count-1 of A kron A (torch tensors, any device):
    row i*a + j (a = rows of A) is A(i,:) kron A(j,:), entry p*c + q =
    A(i,p) A(j,q)."""
    import torch
    a, c = A.shape
    idx = torch.arange(start, start + count, device=A.device, dtype=torch.int64)
    Ai = A.index_select(0, idx // a)
    Aj = A.index_select(0, idx % a)
    prod = (Ai[:, :, None] * Aj[:, None, :]).reshape(count, c * c)
    if out is None:
        return prod
    out.copy_(prod)
    return out

