"""The C-ABI library builds, loads and exports what include/logdet.h declares (no GPU)."""
import ctypes

import pytest

from paper_1811_08057_gb300 import _lib
from paper_1811_08057_gb300 import api


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _lib.header_symbols()
    assert "ld_logdet" in names and "ld_logdet_batched" in names and "ld_logdet_backward" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/logdet.h but not exported"
        assert name in _lib.SIGNATURES, f"{name} has no Python binding"


def test_status_strings(lib):
    for code, name in _lib.STATUS.items():
        assert _lib.ld_status_string(code).startswith(name)
    assert "sm_103a" in _lib.ld_version()


def test_factor_size_matches_documented_layout(lib):
    for mode in range(6):
        f64 = mode in (0, 1)
        for n in [0, 1, 31, 32, 33, 1000]:
            ldf = api._align(max(n, 1), 32)
            es = 8 if f64 else 4
            want = (256 + api._align(n * ldf * es) + 2 * api._align(4 * n) + api._align(8 * n))
            got = _lib.ld_factors_size(n, mode)
            assert got >= want  # the record ends with reserved scratch
            assert got % 256 == 0
    assert _lib.ld_factors_size(-1, 0) == 0
    assert _lib.ld_factors_size(10, 17) == 0


def test_invalid_arguments_rejected_before_any_device_work(lib):
    s = ctypes.c_double()
    l = ctypes.c_double()
    ps, pl = ctypes.addressof(s), ctypes.addressof(l)
    INVALID = 1
    # n < 0, lda < n, NULL matrix, NULL outputs, bad mode, bad dtype
    assert _lib.ld_logdet(0x1000, 0, -1, 4, 0, None, ps, pl) == INVALID
    assert _lib.ld_logdet(0x1000, 0, 8, 4, 0, None, ps, pl) == INVALID
    assert _lib.ld_logdet(None, 0, 8, 8, 0, None, ps, pl) == INVALID
    assert _lib.ld_logdet(0x1000, 0, 8, 8, 0, None, None, pl) == INVALID
    assert _lib.ld_logdet(0x1000, 0, 8, 8, 9, None, ps, pl) == INVALID
    assert _lib.ld_logdet(0x1000, 7, 8, 8, 0, None, ps, pl) == INVALID
    assert _lib.ld_logdet_factor(0x1000, 0, 8, 8, 0, None, None, ps, pl) == INVALID


def test_tuning_table_round_trip(lib):
    assert _lib.ld_get_tuning("blocked_b") in (64, 128)
    assert _lib.ld_set_tuning("blocked_b", 64) == 0
    assert _lib.ld_get_tuning("blocked_b") == 64
    assert _lib.ld_set_tuning("blocked_b", 100) == 1  # not a supported width
    assert _lib.ld_set_tuning("blocked_b", 128) == 0
    for k in range(9):
        assert _lib.ld_set_tuning(f"batched_kb_{k}", 8) == 0
        assert _lib.ld_get_tuning(f"batched_kb_{k}") == 8
        assert _lib.ld_set_tuning(f"batched_kb_{k}", 16) == 0
    assert _lib.ld_set_tuning("batched_kb_9", 8) == 1
    assert _lib.ld_set_tuning("nonsense", 1) == 1
