"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (host only).

The C oracle is built with -fsanitize=address,undefined into a temporary
directory and every pin of test_oracle_mutants.py is run against that build in
a child process (the sanitizer runtime preloaded).  Any out-of-bounds access,
use after free, signed overflow or other undefined behaviour aborts the child.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "mrnmf_oracle.c")

CHILD = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle
import test_oracle_mutants as T
with oracle.substituted({lib!r}):
    res = {{p.__name__: bool(p(oracle)) for p in T.PINS}}
bad = [k for k, v in res.items() if not v]
print("failed pins:", bad)
sys.exit(1 if bad else 0)
"""


def _asan_runtime():
    try:
        path = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True,
                              check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_oracle_pins_under_sanitizers(tmp_path):
    asan = _asan_runtime()
    if asan is None:
        pytest.skip("gcc's AddressSanitizer runtime is not installed")
    lib = str(tmp_path / "liboracle_san.so")
    subprocess.run(["gcc", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                    "-fno-omit-frame-pointer", "-fPIC", "-shared", "-std=c99", "-o", lib, SRC, "-lm"], check=True)
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, tests=HERE, lib=lib)], env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, (out.stdout[-2000:], out.stderr[-4000:])
    assert "runtime error" not in out.stderr and "AddressSanitizer" not in out.stderr, out.stderr[-4000:]


def test_sanitizer_catches_a_planted_overflow(tmp_path):
    # the harness itself: one write past the end of the column-sum output
    # must abort the child with an AddressSanitizer report
    asan = _asan_runtime()
    if asan is None:
        pytest.skip("gcc's AddressSanitizer runtime is not installed")
    text = open(SRC).read()
    site = "        s[j] = sum;\n"
    assert text.count(site) == 1
    src = tmp_path / "oob.c"
    src.write_text(text.replace(site, site + "        s[j + n] = sum;\n"))
    lib = str(tmp_path / "liboob.so")
    subprocess.run(["gcc", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                    "-fno-omit-frame-pointer", "-fPIC", "-shared", "-std=c99", "-o", lib, str(src), "-lm"],
                   check=True)
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:halt_on_error=1")
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, tests=HERE, lib=lib)], env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode != 0 and "heap-buffer-overflow" in out.stderr
