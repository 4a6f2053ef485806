"""The autotuner measures its candidates through the C ABI and applies winners;
results do not depend on the tuning (the batched sweep performs the same
per-element operations for any panel depth)."""
import json

import numpy as np
import pytest
import torch

import workloads
from paper_1811_08057_gb300 import _lib, api, tune

pytestmark = pytest.mark.gpu


def test_batched_results_independent_of_panel_depth():
    mats = [torch.from_numpy(workloads.dense_gaussian(n, seed=n)).cuda() for n in [40, 130, 300]]
    outs = []
    for kb in (8, 16):
        for k in range(9):
            _lib.ld_set_tuning(f"batched_kb_{k}", kb)
        s, l = api.logdet_batched(mats, "f64_plain")
        outs.append((s.clone(), l.clone()))
    for k in range(9):
        _lib.ld_set_tuning(f"batched_kb_{k}", 16)
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_autotune_writes_and_applies_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("LD_TUNE_CACHE", str(tmp_path / "tune.json"))
    entry = tune.autotune(save=True)
    assert entry["blocked_b"] in (64, 128)
    with open(tmp_path / "tune.json") as f:
        data = json.load(f)
    assert torch.cuda.get_device_name(0) in data
    _lib.ld_set_tuning("blocked_b", 64 if entry["blocked_b"] == 128 else 128)
    assert tune.apply()
    assert _lib.ld_get_tuning("blocked_b") == entry["blocked_b"]


def test_blocked_panel_width_64_parity():
    n = 700
    A = workloads.dense_gaussian(n, seed=9, var=1.0 / n) + 2.0 * np.eye(n)
    import oracle
    ref = oracle.logdet(A)
    _lib.ld_set_tuning("blocked_b", 64)
    try:
        for mode in ["f32_3xtf32", "f64_blocked"]:
            s, l = api.logdet(torch.from_numpy(A).cuda(), mode)
            assert float(s) == ref.sign
            tol = 1e-12 if mode == "f64_blocked" else 1e-5
            assert abs(float(l) - ref.logabs) <= tol * max(1.0, abs(ref.logabs))
        Ad, sgn, la, perm = workloads.dyadic_lu(300, seed=1)
        f = api.logdet_factor(torch.from_numpy(Ad).cuda(), "f32_3xtf32")
        assert np.array_equal(f.pivot_labels().cpu().numpy(), perm)
    finally:
        _lib.ld_set_tuning("blocked_b", 128)
