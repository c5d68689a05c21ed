"""The C ABI's host glue under AddressSanitizer and UndefinedBehaviorSanitizer
(no GPU): the library's host code is built with both sanitizers and a child
process drives every argument check, handle creation and destruction, and the
error-string path.  These paths run before any device work, so they run here;
any out-of-bounds access or undefined behaviour aborts the child."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, sys
sys.path.insert(0, {root!r})
from paper_1402_6964_gb300 import mrnmf
lib = mrnmf.load({lib!r})
h = ctypes.c_void_p()
assert lib.mrnmf_create(ctypes.byref(h)) == 0
d = ctypes.c_void_p(16)
sz = ctypes.c_size_t(0)
checks = [
    lib.mrnmf_tsqr_r(h, d, 4, 5, 5, 0, 0, d, None, None),
    lib.mrnmf_tsqr_r(h, d, 1000, 0, 5, 0, 0, d, None, None),
    lib.mrnmf_tsqr_r(h, d, 1000, 257, 300, 0, 0, d, None, None),
    lib.mrnmf_tsqr_r(h, None, 1000, 8, 8, 0, 0, d, None, None),
    lib.mrnmf_tsqr_r(h, d, 1000, 8, 8, 5, 0, d, None, None),
    lib.mrnmf_gauss_project(h, d, 1000, 8, 8, 0, 65, 1, 0, d, None, None),
    lib.mrnmf_tsqr_gp(h, d, 1000, 8, 8, 0, 0, d, None, 70, 1, d, None),
    lib.mrnmf_select_extreme(h, 0, d, 8, d, None, 0, 9, d, None, None),
    lib.mrnmf_select_extreme(h, 7, d, 8, d, None, 0, 3, d, None, None),
    lib.mrnmf_select_extreme(h, 2, None, 8, d, None, 4, 3, d, None, None),
    lib.mrnmf_nnls_h(h, d, 8, d, 0, d, None),
    lib.mrnmf_residual(h, d, 8, d, 9, d, d, None),
    lib.mrnmf_rank_sweep(h, 0, d, 8, d, None, 0, 99, d, d, None),
    lib.mrnmf_stream_push(h, d, 10, 8, None),
    lib.mrnmf_stream_end(h, d, None, None, None),
    lib.mrnmf_stream_state_size(h, ctypes.byref(sz)),
    lib.mrnmf_stream_state_save(h, d, 1 << 20, None),
    lib.mrnmf_stream_state_load(h, d, 1 << 20, None),
    lib.mrnmf_r_svd(h, None, 8, d, d, None),
    lib.mrnmf_gather_columns(h, None, 10, 4, 4, 0, d, 2, d, 2, None),
    lib.mrnmf_full_residual(h, None, 10, 4, 4, 0, d, 2, d, d, None),
    lib.mrnmf_wait_selftest(4, 5000000, d, d, None),
    lib.mrnmf_hh_scalars_selftest(None, d, 10, d, None),
    lib.mrnmf_tc_selftest(d, d, d, 8, 32, 1, None, None),
]
bad = [i for i, c in enumerate(checks) if c != mrnmf.ERR_INVALID_ARG]
msg = lib.mrnmf_last_error_string(h)
lib.mrnmf_destroy(h)
lib.mrnmf_destroy(None)
print("unexpected:", bad, msg)
sys.exit(1 if bad or not msg else 0)
"""


def _asan_runtime():
    try:
        path = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True,
                              check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_abi_host_paths_under_sanitizers(tmp_path):
    asan = _asan_runtime()
    if asan is None:
        pytest.skip("gcc's AddressSanitizer runtime is not installed")
    from paper_1402_6964_gb300 import build
    lib = build.build_sanitized(str(tmp_path / "san"))
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, lib=lib)], env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, (out.stdout[-2000:], out.stderr[-4000:])
    assert "runtime error" not in out.stderr and "AddressSanitizer" not in out.stderr, out.stderr[-4000:]
