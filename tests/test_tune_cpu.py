"""The tuning cache on the host: `tune.apply()` loads this GPU's stored panel
widths into the library's tuning table, and leaves it alone when the cache has
no entry for the GPU (or no file). The GPU name is faked; no device work."""
import json

import pytest

from paper_1811_08057_gb300 import _lib, tune

NAMES = ["blocked_b"] + [f"batched_kb_{k}" for k in range(tune.BUCKETS)]


@pytest.fixture
def saved_table():
    before = {nm: _lib.ld_get_tuning(nm) for nm in NAMES}
    yield before
    for nm, v in before.items():
        assert _lib.ld_set_tuning(nm, v) == 0


def test_apply_loads_cached_entry(tmp_path, monkeypatch, saved_table):
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({
        "Other GPU": {"blocked_b": 128, "batched_kb": {"0": 16}},
        "Fake GB300": {"blocked_b": 64, "batched_kb": {"0": 8, "3": 8, "8": 16}},
    }))
    monkeypatch.setenv("LD_TUNE_CACHE", str(path))
    monkeypatch.setattr(tune, "_gpu_key", lambda device: "Fake GB300")
    for nm in NAMES:  # a known starting point
        assert _lib.ld_set_tuning(nm, 128 if nm == "blocked_b" else 16) == 0
    assert tune.apply() is True
    assert _lib.ld_get_tuning("blocked_b") == 64
    assert _lib.ld_get_tuning("batched_kb_0") == 8
    assert _lib.ld_get_tuning("batched_kb_3") == 8
    assert _lib.ld_get_tuning("batched_kb_8") == 16
    assert _lib.ld_get_tuning("batched_kb_1") == 16  # not in the entry: unchanged


def test_apply_without_entry_changes_nothing(tmp_path, monkeypatch, saved_table):
    monkeypatch.setattr(tune, "_gpu_key", lambda device: "Fake GB300")
    monkeypatch.setenv("LD_TUNE_CACHE", str(tmp_path / "missing.json"))
    assert tune.apply() is False
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"Other GPU": {"blocked_b": 64}}))
    monkeypatch.setenv("LD_TUNE_CACHE", str(path))
    assert tune.apply() is False
    assert {nm: _lib.ld_get_tuning(nm) for nm in NAMES} == saved_table


def test_cache_path_default_and_override(monkeypatch):
    monkeypatch.delenv("LD_TUNE_CACHE", raising=False)
    assert tune.cache_path().endswith("liblogdet/tune.json")
    monkeypatch.setenv("LD_TUNE_CACHE", "/x/y.json")
    assert tune.cache_path() == "/x/y.json"
