"""The tuning table's file form on the host (ld_tune_save / ld_tune_load through
the C ABI; no device work): a round trip restores every entry, and a file with a
bad name or value is rejected as a whole, leaving the table unchanged."""
import pytest

from paper_1811_08057_gb300 import _lib, tune


@pytest.fixture
def saved_table():
    before = tune.table()
    yield before
    for nm, v in before.items():
        assert _lib.ld_set_tuning(nm, v) == 0


def test_save_load_round_trip(tmp_path, saved_table):
    path = str(tmp_path / "t.tune")
    assert _lib.ld_set_tuning("blocked_b", 64) == 0
    assert _lib.ld_set_tuning("blocked_pair_min_n", 12345) == 0
    assert _lib.ld_set_tuning("batched_kb_3", 8) == 0
    assert _lib.ld_set_tuning("batched_threads", 128) == 0
    want = tune.table()
    tune.save(path)
    text = open(path).read().split()
    assert text[0:2] == ["blocked_b", "64"]
    scramble = {"blocked_b": 128, "batched_threads": 256, "rankb_2sm": 0}
    for nm in tune.NAMES:  # scramble, then load
        assert _lib.ld_set_tuning(nm, scramble.get(nm, 16)) == 0
    tune.load(path)
    assert tune.table() == want


@pytest.mark.parametrize("bad", ["blocked_b 96\n", "no_such_entry 1\n", "batched_kb_9 8\n",
                                 "batched_threads 192\n",
                                 "blocked_b 64\nbatched_kb_x 8\n", "blocked_b sixty-four\n"])
def test_bad_file_leaves_table(tmp_path, saved_table, bad):
    path = tmp_path / "bad.tune"
    path.write_text(bad)
    before = tune.table()
    assert _lib.ld_tune_load(str(path)) == 1
    assert tune.table() == before
    assert _lib.ld_tune_load(str(tmp_path / "missing.tune")) == 1


def test_tune_rejects_bad_arguments():
    assert _lib.ld_tune([], 4) == 1
    assert _lib.ld_tune([100, -1], 4) == 1
    assert _lib.ld_tune([100], 99) == 1
