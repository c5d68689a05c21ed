"""The tuning table's file format and lookup (host only, no GPU): the first
matching pass line gives the stream factor, the first matching rows line the
warp leaf's tile height where its form has that height and the CTA fits,
batch lines the waves per family; a malformed file is rejected and leaves the
table unchanged, NULL clears it."""
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


def test_rows_lines_pick_the_warp_leaf_tile_height(mrnmf, tmp_path):
    # built-in heights: 64 rows for n <= 32 (one column per lane; with the
    # projection, since the lane-group leaf serves k = 0 there), 32 for 33..64
    assert [mrnmf.tune_leaf_rows(n, k) for n, k in [(20, 12), (50, 0), (50, 20)]] == [64, 32, 32]
    assert mrnmf.tune_leaf_rows(100, 0) == 0   # not the warp leaf's
    path = _write(tmp_path, "rows 33 64 0 0 64\nrows 1 32 1 64 128\nrows 1 64 0 64 32\n")
    assert mrnmf.tune_load(path) == mrnmf.OK
    assert mrnmf.tune_leaf_rows(50, 0) == 64   # first matching line
    assert mrnmf.tune_leaf_rows(50, 20) == 32  # k = 20 outside [0, 0]: third line
    assert mrnmf.tune_leaf_rows(20, 12) == 128
    assert mrnmf.tune_leaf_rows(20, 0) == 64   # the lane-group leaf's super-tile, whatever the table says
    assert mrnmf.tune_leaf_rows(100, 0) == 0


def test_rows_line_the_form_cannot_take_gives_the_default(mrnmf, tmp_path):
    # 32 rows is not a height of the one-column form, 128 not one of the two-column form
    assert mrnmf.tune_load(_write(tmp_path, "rows 1 32 0 64 32\nrows 33 64 0 64 128\n")) == mrnmf.OK
    assert mrnmf.tune_leaf_rows(20, 12) == 64
    assert mrnmf.tune_leaf_rows(50, 0) == 32
    # n = 64 with 64 projection rows: four 64-row slices need 232 KB of shared memory
    assert mrnmf.tune_load(_write(tmp_path, "rows 33 64 0 64 64\n")) == mrnmf.OK
    assert mrnmf.tune_leaf_rows(64, 0) == 64
    assert mrnmf.tune_leaf_rows(64, 64) == 32


@pytest.mark.parametrize("bad", ["rows 1 8 0 4 48\n", "rows 1 8 4 2 64\n", "rows 8 1 0 4 64\n",
                                 "rows 1 8 -1 4 64\n", "rows 1 8 0 4\n"])
def test_malformed_rows_line_is_rejected(mrnmf, tmp_path, bad):
    assert mrnmf.tune_load(_write(tmp_path, "rows 1 64 0 64 64\n")) == mrnmf.OK
    p = tmp_path / "bad.txt"
    p.write_text(bad)
    assert mrnmf.tune_load(str(p)) == mrnmf.ERR_INVALID_ARG
    assert mrnmf.tune_leaf_rows(50, 0) == 64   # table unchanged


def test_leaf_rows_query_rejects_bad_arguments(mrnmf):
    import ctypes
    lib = mrnmf.load()
    r = ctypes.c_int32(0)
    assert lib.mrnmf_tune_leaf_rows(0, 0, ctypes.byref(r)) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_tune_leaf_rows(10, -1, ctypes.byref(r)) == mrnmf.ERR_INVALID_ARG
    assert lib.mrnmf_tune_leaf_rows(10, 0, None) == mrnmf.ERR_INVALID_ARG


def test_lane_group_leaf_heights_are_fixed(mrnmf, tmp_path):
    # n <= 28 without the projection runs on the lane-group leaf: super-tiles of
    # 32 * 64/S rows (S = 4, 8, 16, 32 lanes a stream), which rows lines do not
    # change; with the projection the warp leaf serves those widths and follows the table
    assert mrnmf.tune_load(_write(tmp_path, "rows 1 32 0 64 128\n")) == mrnmf.OK
    assert [mrnmf.tune_leaf_rows(n, 0) for n in (1, 4, 5, 8, 9, 16, 17, 28)] == [512, 512, 256, 256, 128, 128, 64, 64]
    assert mrnmf.tune_leaf_rows(8, 12) == 128
    assert mrnmf.tune_leaf_rows(25, 16) == 128
    assert mrnmf.tune_leaf_rows(32, 0) == 128   # n = 29..32 without the projection: the warp leaf again
    assert mrnmf.tune_leaf_rows(33, 0) == 32
