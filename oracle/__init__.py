"""FP64 CPU oracle for the TSQR pass and the n-by-n separable step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference``) may import
this package.  The CUDA path in ``paper_1402_6964_gb300`` never imports it and
shares no code with it: the arithmetic lives in ``mrnmf_oracle.c`` (plain C,
built here with gcc) and this module only marshals numpy arrays.

Each wrapper names the passage of Benson, Lee, Rajwa and Gleich (arXiv
1402.6964) that the C routine follows.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrnmf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_NOT_CONVERGED = 4
ERR_RANK = 7


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only: it builds on x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
               "-std=c99", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    d, i64, i32, u64 = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
    P = ctypes.c_void_p
    lib.orc_qr_r.argtypes = [P, i64, i64, i32, P]
    lib.orc_colsum.argtypes = [P, i64, i64, i32, P]
    lib.orc_philox4x32_10.argtypes = [P, P, P]
    lib.orc_gauss_entry.argtypes = [u64, i64, i32]
    lib.orc_gauss_entry.restype = d
    lib.orc_gauss_matrix.argtypes = [u64, i64, i64, i32, P]
    lib.orc_gauss_project.argtypes = [P, i64, i64, i32, i32, u64, i64, P]
    lib.orc_nnls.argtypes = [P, P, d, i32, P]
    lib.orc_nnls_h.argtypes = [P, i32, i32, P, i32, P]
    lib.orc_residual.argtypes = [P, i32, i32, P, i32, P, P]
    lib.orc_spa.argtypes = [P, i32, i32, P, i32, P, P]
    lib.orc_xray.argtypes = [P, i32, i32, i32, P, P]
    lib.orc_gp_select.argtypes = [P, i32, i32, P, i32, P, P, P, P, P]
    lib.orc_r_svd.argtypes = [P, i32, P, P]
    return lib


@contextlib.contextmanager
def substituted(path: str):
    """Route every wrapper to another build of the oracle's source (the pin
    tests use this to check that a planted mistake fails a pin)."""
    global _lib
    lib = _bind(ctypes.CDLL(path))
    with _lock:
        saved = _lib
        _lib = lib
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def qr_r(X) -> np.ndarray:
    """R factor of the thin QR of X (Sec. 3.1), unblocked Householder, diag(R) >= 0."""
    X = _f64(X)
    m, n = X.shape
    R = np.zeros((n, n), np.float64)
    st = _load().orc_qr_r(_ptr(X), m, n, n, _ptr(R))
    if st != OK:
        raise RuntimeError(f"orc_qr_r failed: {st}")
    return R


def colsum(X) -> np.ndarray:
    """Column sums (= l1 column norms of a nonnegative X; Sec. 2.1, Sec. 3.3), Kahan-summed."""
    X = _f64(X)
    m, n = X.shape
    s = np.zeros(n, np.float64)
    _load().orc_colsum(_ptr(X), m, n, n, _ptr(s))
    return s


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def gauss_matrix(seed: int, row0: int, rows: int, k: int) -> np.ndarray:
    """Rows row0..row0+rows-1 of the m-by-k Gaussian G (Sec. 2.3, Algorithm 1)."""
    G = np.zeros((rows, k), np.float64)
    _load().orc_gauss_matrix(seed, row0, rows, k, _ptr(G))
    return G


def gauss_project(X, k: int, seed: int, row0: int = 0) -> np.ndarray:
    """GX = G^T X (k-by-n), summed row by row (Sec. 3.2, Algorithm 1)."""
    X = _f64(X)
    m, n = X.shape
    GX = np.zeros((k, n), np.float64)
    _load().orc_gauss_project(_ptr(X), m, n, n, k, seed, row0, _ptr(GX))
    return GX


def nnls(AtA, Atb, btb: float):
    """Lawson-Hanson NNLS on the normal equations (Sec. 2.4). Returns (x, status)."""
    AtA = _f64(AtA)
    Atb = _f64(Atb)
    r = Atb.shape[0]
    x = np.zeros(r, np.float64)
    st = _load().orc_nnls(_ptr(AtA), _ptr(Atb), float(btb), r, _ptr(x))
    return x, st


def nnls_h(R, K):
    """H(:,i) = argmin_{y>=0} ||R(:,K) y - R(:,i)|| for every column i (Sec. 2.4).

    R may be the n-by-n factor or X itself (rows-by-n).  Returns (H, status).
    """
    R = _f64(R)
    rows, n = R.shape
    K = np.ascontiguousarray(K, dtype=np.int32)
    r = K.shape[0]
    H = np.zeros((r, n), np.float64)
    st = _load().orc_nnls_h(_ptr(R), rows, n, _ptr(K), r, _ptr(H))
    return H, st


def residual(R, K, H):
    """(||R - R(:,K)H||_F, ||R - R(:,K)H||_F^2 / ||R||_F^2)  (Sec. 2.4, Sec. 4)."""
    R = _f64(R)
    rows, n = R.shape
    K = np.ascontiguousarray(K, dtype=np.int32)
    H = _f64(H)
    out = np.zeros(2, np.float64)
    _load().orc_residual(_ptr(R), rows, n, _ptr(K), K.shape[0], _ptr(H), _ptr(out))
    return float(out[0]), float(out[1])


def spa(Y, colsum_, r: int):
    """SPA on Y D^-1 (Sec. 2.1).  Returns (K, gap); gap[t] = -1 marks a step
    whose best residual is zero to rounding."""
    Y = _f64(Y)
    rows, n = Y.shape
    s = _f64(colsum_)
    K = np.zeros(r, np.int32)
    gap = np.zeros(r, np.float64)
    st = _load().orc_spa(_ptr(Y), rows, n, _ptr(s), r, _ptr(K), _ptr(gap))
    if st != OK:
        raise RuntimeError(f"orc_spa failed: {st}")
    return K, gap


def xray(Y, r: int):
    """Greedy XRAY (Sec. 2.1).  Returns (K, gap, status)."""
    Y = _f64(Y)
    rows, n = Y.shape
    K = np.zeros(r, np.int32)
    gap = np.zeros(r, np.float64)
    st = _load().orc_xray(_ptr(Y), rows, n, r, _ptr(K), _ptr(gap))
    return K, gap, st


def gp_select(GX, colsum_, r: int):
    """Gaussian-projection selection (Sec. 2.3, Sec. 3.3).

    Returns (K, candidates, gap per candidate); the gap of a candidate is the
    relative margin of the row max / min that added it."""
    GX = _f64(GX)
    k, n = GX.shape
    s = _f64(colsum_)
    K = np.zeros(r, np.int32)
    cand = np.zeros(2 * k, np.int32)
    nc = ctypes.c_int(0)
    gap = np.zeros(2 * k, np.float64)
    cgap = np.zeros(2 * k, np.float64)
    _load().orc_gp_select(_ptr(GX), k, n, _ptr(s), r, _ptr(K), _ptr(cand), ctypes.byref(nc), _ptr(gap),
                          _ptr(cgap))
    return K, cand[: nc.value].copy(), cgap[: nc.value].copy()


def r_svd(R):
    """Sigma V' of a square R by one-sided Jacobi (Sec. 2.2; the R-SVD of
    Sec. 3.1): (sigma descending, SVt with row i = sigma_i v_i', status)."""
    R = _f64(R)
    n = R.shape[0]
    sig = np.zeros(n)
    S = np.zeros((n, n))
    st = _load().orc_r_svd(_ptr(R), n, _ptr(sig), _ptr(S))
    return sig, S, st
