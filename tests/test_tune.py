"""The tuning table's file format and lookup (host only, no GPU): the first
matching pass line gives the stream factor, batch lines the waves per family,
a malformed file is rejected and leaves the table unchanged, NULL clears it."""
import pytest


@pytest.fixture()
def mrnmf(tmp_path):
    from paper_1402_6964_gb300 import build, mrnmf as m
    build.build()
    m.tune_load(None)
    yield m
    m.tune_load(None)


def _write(tmp_path, text):
    p = tmp_path / "tune.txt"
    p.write_text(text)
    return str(p)


def test_lookup_follows_the_first_matching_line(mrnmf, tmp_path):
    path = _write(tmp_path, "# comment\npass 33 64 20 24 0.5\npass 1 256 0 64 2\n\nbatch 3 16\nbatch 1 4\n")
    assert mrnmf.tune_load(path) == mrnmf.OK
    assert mrnmf.tune_query(50, 2 ** 22) == (0.5, [4.0, 0.0, 16.0])   # log2 m = 22 in [20, 24)
    assert mrnmf.tune_query(50, 2 ** 24)[0] == 2.0                    # [20, 24) excludes 24
    assert mrnmf.tune_query(64, 2 ** 20)[0] == 0.5
    assert mrnmf.tune_query(65, 2 ** 22)[0] == 2.0
    assert mrnmf.tune_query(50, 0)[0] == 1.0                          # unknown m: no tuning


@pytest.mark.parametrize("bad", ["pass 33 64 20 24\n", "pass 64 33 20 24 1\n", "pass 1 8 4 2 1\n",
                                 "pass 1 8 0 4 0\n", "batch 4 8\n", "batch 1 0.1\n", "steps 3\n"])
def test_malformed_table_is_rejected_and_leaves_the_table(mrnmf, tmp_path, bad):
    good = _write(tmp_path, "pass 1 256 0 64 0.25\n")
    assert mrnmf.tune_load(good) == mrnmf.OK
    p = tmp_path / "bad.txt"
    p.write_text(bad)
    assert mrnmf.tune_load(str(p)) == mrnmf.ERR_INVALID_ARG
    assert mrnmf.tune_query(10, 1000)[0] == 0.25


def test_missing_file_and_clear(mrnmf, tmp_path):
    assert mrnmf.tune_load(str(tmp_path / "absent.txt")) == mrnmf.ERR_INVALID_ARG
    assert mrnmf.tune_load(_write(tmp_path, "pass 1 256 0 64 3\n")) == mrnmf.OK
    assert mrnmf.tune_query(100, 10 ** 6)[0] == 3.0
    assert mrnmf.tune_load(None) == mrnmf.OK
    assert mrnmf.tune_query(100, 10 ** 6) == (1.0, [0.0, 0.0, 0.0])
