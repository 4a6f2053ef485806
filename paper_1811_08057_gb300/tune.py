"""Autotuner for the library's tuning table (ld_set_tuning).

Times candidate settings through the C ABI on synthetic inputs of the target
shapes and keeps the fastest:
  blocked_b          panel width of the blocked sweep (64 or 128), timed on an
                     N x N dense iid N(0, 1/N) matrix in the requested mode
  batched_kb_<k>     panel depth of the batched sweep (8 or 16) for matrices with
                     n in [64k, 64k + 63], timed on a batch of that size class
Results are cached as JSON (path from LD_TUNE_CACHE, default
~/.cache/liblogdet/tune.json) keyed by GPU name; `apply()` loads the cache into
the library, `autotune()` measures and stores.
"""
from __future__ import annotations

import json
import os

import torch

from . import _lib
from . import api

BUCKETS = 9


def cache_path() -> str:
    return os.environ.get("LD_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "liblogdet", "tune.json"))


def _gpu_key(device) -> str:
    return torch.cuda.get_device_name(device)


def _time(fn, reps=3, warmup=1):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_blocked(N=4096, mode="f32_3xtf32", device="cuda", seed=0):
    g = torch.Generator(device=device).manual_seed(seed)
    A = torch.randn(N, N, generator=g, device=device, dtype=torch.float32) / N ** 0.5
    times = {}
    for b in (64, 128):
        _lib.check("ld_set_tuning", _lib.ld_set_tuning("blocked_b", b))
        times[b] = _time(lambda: api.logdet(A, mode))
    best = min(times, key=times.get)
    _lib.check("ld_set_tuning", _lib.ld_set_tuning("blocked_b", best))
    return best, times


def tune_batched(count_per_class=256, device="cuda", seed=0):
    choice, detail = {}, {}
    g = torch.Generator(device=device).manual_seed(seed)
    for k in range(BUCKETS):
        n = min(64 * k + 48, 512) if k < BUCKETS - 1 else 512
        n = max(n, 16)
        X = torch.randn(count_per_class, 2 * n, n, generator=g, device=device)
        S = torch.bmm(X.transpose(1, 2), X) / (2 * n)
        S.diagonal(dim1=1, dim2=2).add_(1e-2)
        batch = api.BatchedInputs(list(S))
        times = {}
        for kb in (8, 16):
            _lib.check("ld_set_tuning", _lib.ld_set_tuning(f"batched_kb_{k}", kb))
            times[kb] = _time(lambda: api.logdet_batched(batch, "f32_plain"))
        best = min(times, key=times.get)
        _lib.check("ld_set_tuning", _lib.ld_set_tuning(f"batched_kb_{k}", best))
        choice[k] = best
        detail[k] = {"n": n, "ms": times}
    return choice, detail


def autotune(device=0, save=True):
    """Measure every tunable on this GPU, apply the winners, store them."""
    dev = torch.device("cuda", device)
    b, bt = tune_blocked(device=dev)
    kb, kbt = tune_batched(device=dev)
    entry = {"blocked_b": b, "batched_kb": {str(k): v for k, v in kb.items()},
             "timings": {"blocked": {str(k): v for k, v in bt.items()},
                         "batched": {str(k): {"n": v["n"], "ms": {str(a): t for a, t in v["ms"].items()}}
                                     for k, v in kbt.items()}}}
    if save:
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        data = {}
        if os.path.exists(path):
            with open(path) as f:
                data = json.load(f)
        data[_gpu_key(dev)] = entry
        with open(path, "w") as f:
            json.dump(data, f, indent=1)
    return entry


def apply(device=0) -> bool:
    """Load this GPU's cached settings into the library (False if none cached)."""
    path = cache_path()
    if not os.path.exists(path):
        return False
    with open(path) as f:
        data = json.load(f)
    entry = data.get(_gpu_key(torch.device("cuda", device)))
    if not entry:
        return False
    _lib.check("ld_set_tuning", _lib.ld_set_tuning("blocked_b", int(entry["blocked_b"])))
    for k, v in entry.get("batched_kb", {}).items():
        _lib.check("ld_set_tuning", _lib.ld_set_tuning(f"batched_kb_{int(k)}", int(v)))
    return True
