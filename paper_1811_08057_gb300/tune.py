"""Thin driver of the library's autotuner (ld_tune, ld_tune_save, ld_tune_load).

The timing loop, the candidates and the cache file live in the C library
(csrc/tune.cu): ld_tune times panel widths and paired updates for the blocked
modes, and the batched panel depth per size class for the plain modes, on
synthetic matrices of the caller's sizes, and applies the fastest. With
LD_TUNE_CACHE set to a directory, the table is stored there per GPU name and
loaded by the library on first use.
"""
from __future__ import annotations

from . import _lib

BUCKETS = 9
NAMES = (["blocked_b", "blocked_pair_min_n", "rankb_2sm", "batched_threads"] +
         [f"batched_kb_{k}" for k in range(BUCKETS)])


def table() -> dict:
    """The library's tuning table."""
    return {nm: _lib.ld_get_tuning(nm) for nm in NAMES}


def autotune(sizes, mode="f32_3xtf32", stream=None) -> dict:
    """Times the candidates for these matrix sizes in `mode`, applies the winners
    (and stores them when LD_TUNE_CACHE is set); returns the table."""
    _lib.check("ld_tune", _lib.ld_tune(list(sizes), _lib.MODES[mode], stream))
    return table()


def save(path=None):
    _lib.check("ld_tune_save", _lib.ld_tune_save(path))


def load(path=None):
    _lib.check("ld_tune_load", _lib.ld_tune_load(path))
