"""Thin ctypes binding of libmrnmf.so (include/mrnmf.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are torch CUDA tensors; torch is used for device memory and
streams and nothing else.  If the library is missing the import of a function
raises -- there is no CPU fallback.

Function names follow the C ABI without the ``mrnmf_`` prefix.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmrnmf.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_NO_MEMORY, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_BAD_INPUT, ERR_RANK_DEFICIENT = range(8)
F32, F64 = 0, 1
PREC = {"auto": 0, "fp64": 1, "fp32": 2, "tf32x3": 3, "bf16": 4, "tf32": 5}
METHOD = {"spa": 0, "xray": 1, "gp": 2}

EXPORTS = [
    "mrnmf_create", "mrnmf_destroy", "mrnmf_last_error_string", "mrnmf_sync_status", "mrnmf_tsqr_r",
    "mrnmf_gauss_project", "mrnmf_gauss_project_tc", "mrnmf_tsqr_gp", "mrnmf_select_extreme", "mrnmf_nnls_h", "mrnmf_residual",
    "mrnmf_stream_begin", "mrnmf_stream_push", "mrnmf_stream_end", "mrnmf_factorize_host",
    "mrnmf_profile_events", "mrnmf_kernel_launches", "mrnmf_tsqr_r_noalloc", "mrnmf_tc_selftest", "mrnmf_wait_selftest", "mrnmf_hh_scalars_selftest",
    "mrnmf_rank_sweep", "mrnmf_tsqr_r_batched", "mrnmf_gather_columns", "mrnmf_full_residual",
    "mrnmf_r_svd", "mrnmf_stream_state_size", "mrnmf_stream_state_save", "mrnmf_stream_state_load",
    "mrnmf_tune_load", "mrnmf_tune_query", "mrnmf_tune_leaf_rows",
]


class Problem(ctypes.Structure):
    """mrnmf_problem: one member of a batched pass."""
    _fields_ = [("X", ctypes.c_void_p), ("m", ctypes.c_int64), ("ldx", ctypes.c_int64), ("n", ctypes.c_int32),
                ("R", ctypes.c_void_p), ("colsum", ctypes.c_void_p)]


class MrnmfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mrnmf status {status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libmrnmf.so (built in-tree by paper_1402_6964_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None and path == LIB_PATH:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        st = ctypes.c_int
        sig = {
            "mrnmf_create": ([ctypes.POINTER(P)], st),
            "mrnmf_destroy": ([P], None),
            "mrnmf_last_error_string": ([P], ctypes.c_char_p),
            "mrnmf_sync_status": ([P, P], st),
            "mrnmf_tsqr_r": ([P, P, i64, i32, i64, i32, i32, P, P, P], st),
            "mrnmf_gauss_project": ([P, P, i64, i32, i64, i32, i32, u64, i64, P, P, P], st),
            "mrnmf_gauss_project_tc": ([P, P, i64, i32, i64, i32, u64, i64, i32, P, P, P], st),
            "mrnmf_tsqr_gp": ([P, P, i64, i32, i64, i32, i32, P, P, i32, u64, P, P], st),
            "mrnmf_select_extreme": ([P, i32, P, i32, P, P, i32, i32, P, P, P], st),
            "mrnmf_nnls_h": ([P, P, i32, P, i32, P, P], st),
            "mrnmf_residual": ([P, P, i32, P, i32, P, P, P], st),
            "mrnmf_stream_begin": ([P, i32, i32, i32, i32, u64, P], st),
            "mrnmf_stream_push": ([P, P, i64, i64, P], st),
            "mrnmf_stream_end": ([P, P, P, P, P], st),
            "mrnmf_factorize_host": ([P, P, i64, i32, i64, i32, i32, i32, i32, u64, P, P, P, P, P], st),
            "mrnmf_profile_events": ([P, P, P], st),
            "mrnmf_kernel_launches": ([], ctypes.c_uint64),
            "mrnmf_tsqr_r_noalloc": ([P, i64, i32, i64, P, P, P, P], st),
            "mrnmf_tc_selftest": ([P, P, P, i32, i32, i32, P, P], st),
            "mrnmf_wait_selftest": ([i32, ctypes.c_int64, P, P, P], st),
            "mrnmf_hh_scalars_selftest": ([P, P, i64, P, P], st),
            "mrnmf_rank_sweep": ([P, i32, P, i32, P, P, i32, i32, P, P, P], st),
            "mrnmf_tsqr_r_batched": ([P, P, i32, P], st),
            "mrnmf_gather_columns": ([P, P, i64, i32, i64, i32, P, i32, P, i64, P], st),
            "mrnmf_full_residual": ([P, P, i64, i32, i64, i32, P, i32, P, P, P], st),
            "mrnmf_r_svd": ([P, P, i32, P, P, P], st),
            "mrnmf_stream_state_size": ([P, ctypes.POINTER(ctypes.c_size_t)], st),
            "mrnmf_stream_state_save": ([P, P, ctypes.c_size_t, P], st),
            "mrnmf_stream_state_load": ([P, P, ctypes.c_size_t, P], st),
            "mrnmf_tune_load": ([ctypes.c_char_p], st),
            "mrnmf_tune_query": ([i32, i64, P, P], st),
            "mrnmf_tune_leaf_rows": ([i32, i32, P], st),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        if path == LIB_PATH:
            _lib = lib
        return lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(X):
    import torch
    if X.dtype == torch.float32:
        return F32
    if X.dtype == torch.float64:
        return F64
    raise TypeError("X must be float32 or float64")


def _check_X(X):
    if not X.is_cuda:
        raise ValueError("X must be a CUDA tensor (use factorize_host for host data)")
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be 2-D with unit column stride (row-major)")


def kernel_launches() -> int:
    """Kernels launched by libmrnmf in this process so far."""
    return int(load().mrnmf_kernel_launches())


def tsqr_r_noalloc(X, R, colsum=None, status=None, stream=None) -> int:
    """mrnmf_tsqr_r_noalloc: R (and colsum) of a float32 CUDA X into caller
    buffers, with no device allocation inside the library.  `status` is a
    one-element int32 CUDA tensor and is required (None is passed as NULL,
    which the library rejects).  Returns the C status of the call; device-side
    errors land in `status`."""
    _check_X(X)
    m, n = X.shape
    return int(load().mrnmf_tsqr_r_noalloc(_ptr(X), m, n, X.stride(0), _ptr(R), _ptr(colsum), _ptr(status),
                                           _stream(stream)))


def tune_load(path) -> int:
    """mrnmf_tune_load: replace the process-wide tuning table with the file at
    `path` (None clears it).  Returns the C status."""
    return int(load().mrnmf_tune_load(None if path is None else os.fsencode(path)))


def tune_query(n: int, m: int):
    """mrnmf_tune_query: (stream factor for a pass of n columns over m rows,
    [waves planned for batch families 1..3, 0 = built-in default])."""
    f = ctypes.c_double(0.0)
    w = (ctypes.c_double * 3)()
    st = int(load().mrnmf_tune_query(n, m, ctypes.byref(f), w))
    if st != OK:
        raise MrnmfError(st, "tune query")
    return f.value, list(w)


def tune_leaf_rows(n: int, k: int = 0) -> int:
    """mrnmf_tune_leaf_rows: tile height of the warp leaf for a binary32 pass
    of n columns with k projection rows (0 where that leaf does not serve it)."""
    r = ctypes.c_int32(0)
    st = int(load().mrnmf_tune_leaf_rows(n, k, ctypes.byref(r)))
    if st != OK:
        raise MrnmfError(st, "tune leaf rows")
    return r.value


def tc_selftest(A, B, kind="tf32x3", status=None, stream=None):
    """D = A B^T on the tcgen05 tensor cores (A 128-by-K, B N-by-K, float32 CUDA)."""
    import torch
    N, K = B.shape
    D = torch.empty((A.shape[0], N), dtype=torch.float32, device=A.device)
    code = {"tf32": 0, "tf32x3": 1, "bf16": 2}[kind]
    st = int(load().mrnmf_tc_selftest(_ptr(A), _ptr(B), _ptr(D), N, K, code, _ptr(status), _stream(stream)))
    if st != OK:
        raise MrnmfError(st, "tc_selftest rejected its arguments")
    return D


def hh_scalars_selftest(alpha, sigma, stream=None):
    """The leaves' Householder scalars and the IEEE ones for float32 CUDA
    `alpha`, `sigma`: a (count, 8) tensor, columns beta, d, 1/beta, 1/d of
    the leaves, then of the IEEE operations."""
    import torch
    out = torch.empty((alpha.numel(), 8), dtype=torch.float32, device=alpha.device)
    st = int(load().mrnmf_hh_scalars_selftest(_ptr(alpha), _ptr(sigma), alpha.numel(), _ptr(out), _stream(stream)))
    if st != OK:
        raise MrnmfError(st, "hh_scalars_selftest rejected its arguments")
    return out


def wait_selftest(missing, limit_ns, device="cuda", stream=None):
    """Failure injection on the leaf's bounded wait: returns the per-warp
    outcome codes (0 completed, 1 ran out, 2 abandoned) and the status word,
    both as device int32 tensors."""
    import torch
    out = torch.full((4,), -1, dtype=torch.int32, device=device)
    status = torch.zeros(1, dtype=torch.int32, device=device)
    st = int(load().mrnmf_wait_selftest(missing, limit_ns, _ptr(out), _ptr(status), _stream(stream)))
    if st != OK:
        raise MrnmfError(st, "wait_selftest rejected its arguments")
    return out, status


class Handle:
    """Owns an mrnmf_handle (its device workspace and status word)."""

    def __init__(self):
        self._lib = load()
        h = ctypes.c_void_p()
        self._check(self._lib.mrnmf_create(ctypes.byref(h)), None)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self._lib.mrnmf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, status, h):
        if status != OK:
            msg = self._lib.mrnmf_last_error_string(h).decode() if h else "invalid argument"
            raise MrnmfError(status, msg)

    def check(self, status):
        self._check(status, self.h)

    def profile_events(self, start=None, stop=None):
        """Record torch.cuda.Event `start`/`stop` around the leaf kernel of later passes."""
        self.check(self._lib.mrnmf_profile_events(
            self.h, ctypes.c_void_p(start.cuda_event) if start is not None else None,
            ctypes.c_void_p(stop.cuda_event) if stop is not None else None))

    def sync(self, stream=None):
        """Wait for the stream and raise on any error the kernels recorded."""
        self.check(self._lib.mrnmf_sync_status(self.h, _stream(stream)))

    # ------------------------------------------------------------- the pass
    def tsqr_r(self, X, prec="auto", stream=None, colsum=True):
        import torch
        _check_X(X)
        m, n = X.shape
        R = torch.empty((n, n), dtype=torch.float64, device=X.device)
        cs = torch.empty(n, dtype=torch.float64, device=X.device) if colsum else None
        self.check(self._lib.mrnmf_tsqr_r(self.h, _ptr(X), m, n, X.stride(0), _dtype_code(X), PREC[prec],
                                          _ptr(R), _ptr(cs), _stream(stream)))
        return R, cs

    def gauss_project(self, X, k, seed, row_offset=0, stream=None):
        import torch
        _check_X(X)
        m, n = X.shape
        GX = torch.empty((k, n), dtype=torch.float64, device=X.device)
        cs = torch.empty(n, dtype=torch.float64, device=X.device)
        self.check(self._lib.mrnmf_gauss_project(self.h, _ptr(X), m, n, X.stride(0), _dtype_code(X), k, seed,
                                                 row_offset, _ptr(GX), _ptr(cs), _stream(stream)))
        return GX, cs

    def gauss_project_tc(self, X, k, seed, form="bf16", row_offset=0, stream=None):
        """mrnmf_gauss_project_tc: G'X on the tensor cores, form "bf16" or "tf32x3"."""
        import torch
        _check_X(X)
        m, n = X.shape
        GX = torch.empty((k, n), dtype=torch.float64, device=X.device)
        cs = torch.empty(n, dtype=torch.float64, device=X.device)
        self.check(self._lib.mrnmf_gauss_project_tc(self.h, _ptr(X), m, n, X.stride(0), k, seed, row_offset,
                                                    PREC[form], _ptr(GX), _ptr(cs), _stream(stream)))
        return GX, cs

    def tsqr_gp(self, X, k, seed, prec="auto", stream=None, out=None):
        import torch
        _check_X(X)
        m, n = X.shape
        if out is None:
            R = torch.empty((n, n), dtype=torch.float64, device=X.device)
            cs = torch.empty(n, dtype=torch.float64, device=X.device)
            GX = torch.empty((max(k, 1), n), dtype=torch.float64, device=X.device)
        else:
            R, cs, GX = out
        self.check(self._lib.mrnmf_tsqr_gp(self.h, _ptr(X), m, n, X.stride(0), _dtype_code(X), PREC[prec],
                                           _ptr(R), _ptr(cs), k, seed, _ptr(GX) if k > 0 else None,
                                           _stream(stream)))
        return R, cs, (GX if k > 0 else None)

    # -------------------------------------------------------- n-by-n step
    def select_extreme(self, method, R=None, colsum=None, GX=None, r=1, stream=None, out=None):
        import torch
        ref = R if R is not None else GX
        n = ref.shape[1]
        k = GX.shape[0] if GX is not None else 0
        if out is None:
            K = torch.empty(r, dtype=torch.int32, device=ref.device)
            gap = torch.empty(r, dtype=torch.float64, device=ref.device)
        else:
            K, gap = out
        self.check(self._lib.mrnmf_select_extreme(self.h, METHOD[method], _ptr(R), n, _ptr(colsum), _ptr(GX), k, r,
                                                  _ptr(K), _ptr(gap), _stream(stream)))
        return K, gap

    def nnls_h(self, R, K, stream=None, out=None):
        import torch
        n = R.shape[1]
        r = K.shape[0]
        H = torch.empty((r, n), dtype=torch.float64, device=R.device) if out is None else out
        self.check(self._lib.mrnmf_nnls_h(self.h, _ptr(R), n, _ptr(K), r, _ptr(H), _stream(stream)))
        return H

    def residual(self, R, K, H, stream=None, out=None):
        import torch
        n = R.shape[1]
        o = torch.empty(2, dtype=torch.float64, device=R.device) if out is None else out
        self.check(self._lib.mrnmf_residual(self.h, _ptr(R), n, _ptr(K), K.shape[0], _ptr(H), _ptr(o),
                                            _stream(stream)))
        return o

    def r_svd(self, R, stream=None):
        """(sigma descending, Sigma V') of the n-by-n R (Sec. 2.2's R-SVD form)."""
        import torch
        n = R.shape[1]
        sig = torch.empty(n, dtype=torch.float64, device=R.device)
        SVt = torch.empty((n, n), dtype=torch.float64, device=R.device)
        self.check(self._lib.mrnmf_r_svd(self.h, _ptr(R), n, _ptr(sig), _ptr(SVt), _stream(stream)))
        return sig, SVt

    def gather_columns(self, X, K, stream=None, out=None):
        """W = X(:, K) (a second read of X)."""
        import torch
        _check_X(X)
        m, n = X.shape
        r = K.shape[0]
        W = torch.empty((m, r), dtype=X.dtype, device=X.device) if out is None else out
        self.check(self._lib.mrnmf_gather_columns(self.h, _ptr(X), m, n, X.stride(0), _dtype_code(X), _ptr(K), r,
                                                  _ptr(W), W.stride(0), _stream(stream)))
        return W

    def full_residual(self, X, K, H, stream=None, out=None):
        """(||X - X(:,K)H||_F, ||X - X(:,K)H||_F^2 / ||X||_F^2) from X itself (a second read)."""
        import torch
        _check_X(X)
        m, n = X.shape
        o = torch.empty(2, dtype=torch.float64, device=X.device) if out is None else out
        self.check(self._lib.mrnmf_full_residual(self.h, _ptr(X), m, n, X.stride(0), _dtype_code(X), _ptr(K),
                                                 K.shape[0], _ptr(H), _ptr(o), _stream(stream)))
        return o

    def rank_sweep(self, method, R=None, colsum=None, GX=None, r_max=1, stream=None):
        """(K for r_max, curve[r-1] = (abs, rel) residual for r = 1..r_max)."""
        import torch
        ref = R if R is not None else GX
        n = ref.shape[1]
        k = GX.shape[0] if GX is not None else 0
        K = torch.empty(r_max, dtype=torch.int32, device=ref.device)
        curve = torch.empty((r_max, 2), dtype=torch.float64, device=ref.device)
        self.check(self._lib.mrnmf_rank_sweep(self.h, METHOD[method], _ptr(R), n, _ptr(colsum), _ptr(GX), k, r_max,
                                              _ptr(K), _ptr(curve), _stream(stream)))
        return K, curve

    def tsqr_r_batched(self, Xs, outs=None, stream=None):
        """R and colsum of every float32 CUDA matrix in Xs, one batched pass.
        outs: optional list of (R, colsum) tensors to fill (reused across calls)."""
        import torch
        if outs is None:
            outs = [(torch.empty((X.shape[1], X.shape[1]), dtype=torch.float64, device=X.device),
                     torch.empty(X.shape[1], dtype=torch.float64, device=X.device)) for X in Xs]
        arr = (Problem * len(Xs))()
        for i, (X, (R, cs)) in enumerate(zip(Xs, outs)):
            _check_X(X)
            if X.dtype != torch.float32:
                raise TypeError("batched pass takes float32")
            arr[i] = Problem(X.data_ptr(), X.shape[0], X.stride(0), X.shape[1], R.data_ptr(),
                             cs.data_ptr() if cs is not None else None)
        self._batch = arr  # keep the descriptors alive
        self.check(self._lib.mrnmf_tsqr_r_batched(self.h, ctypes.cast(arr, ctypes.c_void_p), len(Xs),
                                                  _stream(stream)))
        return outs

    # ------------------------------------------------------------ streaming
    def stream_begin(self, n, dtype="f32", prec="auto", k=0, seed=0, stream=None):
        self.check(self._lib.mrnmf_stream_begin(self.h, n, F64 if dtype == "f64" else F32, PREC[prec], k, seed,
                                                _stream(stream)))

    def stream_push(self, X, stream=None):
        _check_X(X)
        self.check(self._lib.mrnmf_stream_push(self.h, _ptr(X), X.shape[0], X.stride(0), _stream(stream)))

    def stream_state_save(self, stream=None) -> bytes:
        """Checkpoint of the open stream (host bytes)."""
        sz = ctypes.c_size_t(0)
        self.check(self._lib.mrnmf_stream_state_size(self.h, ctypes.byref(sz)))
        buf = ctypes.create_string_buffer(sz.value)
        self.check(self._lib.mrnmf_stream_state_save(self.h, buf, sz.value, _stream(stream)))
        return buf.raw

    def stream_state_load(self, state: bytes, stream=None):
        """Restore a checkpoint into a stream begun with the same parameters."""
        buf = ctypes.create_string_buffer(state, len(state))
        self.check(self._lib.mrnmf_stream_state_load(self.h, buf, len(state), _stream(stream)))

    def stream_end(self, n, k=0, device="cuda", stream=None):
        import torch
        R = torch.empty((n, n), dtype=torch.float64, device=device)
        cs = torch.empty(n, dtype=torch.float64, device=device)
        GX = torch.empty((max(k, 1), n), dtype=torch.float64, device=device)
        self.check(self._lib.mrnmf_stream_end(self.h, _ptr(R), _ptr(cs), _ptr(GX) if k > 0 else None,
                                              _stream(stream)))
        return R, cs, (GX if k > 0 else None)

    # ------------------------------------------------- host end-to-end path
    def factorize_host(self, X, r, method="spa", k=0, seed=0, prec="auto", stream=None, want_R=False):
        """X: host float32 array (numpy, or a CPU torch tensor, ideally pinned)."""
        if hasattr(X, "numpy"):
            if X.is_cuda:
                raise ValueError("factorize_host takes host memory")
            xp = ctypes.c_void_p(X.data_ptr())
            m, n = X.shape
            ldx = X.stride(0)
        else:
            X = np.ascontiguousarray(X, dtype=np.float32)
            xp = _np_ptr(X)
            m, n = X.shape
            ldx = n
        K = np.zeros(r, np.int32)
        H = np.zeros((r, n), np.float64)
        res = np.zeros(2, np.float64)
        R = np.zeros((n, n), np.float64) if want_R else None
        self.check(self._lib.mrnmf_factorize_host(self.h, xp, m, n, ldx, PREC[prec], METHOD[method], r, k, seed,
                                                  _np_ptr(K), _np_ptr(H), _np_ptr(res), _np_ptr(R),
                                                  _stream(stream)))
        return K, H, res, R
