"""The autotuner through the C ABI (ld_tune): it picks candidates the launchers
accept, stores the table under LD_TUNE_CACHE, and a fresh process loads it on
first use; results do not depend on the tuning where the operations are the same
(the batched sweep performs the same per-element operations for any panel depth)."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import workloads
from paper_1811_08057_gb300 import _lib, api, tune

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def saved_table():
    before = tune.table()
    yield before
    for nm, v in before.items():
        assert _lib.ld_set_tuning(nm, v) == 0


def test_batched_results_independent_of_panel_depth(saved_table):
    mats = [torch.from_numpy(workloads.dense_gaussian(n, seed=n)).cuda() for n in [40, 130, 300]]
    outs = []
    for kb in (8, 16):
        for k in range(9):
            _lib.ld_set_tuning(f"batched_kb_{k}", kb)
        s, l = api.logdet_batched(mats, "f64_plain")
        outs.append((s.clone(), l.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_batched_results_independent_of_cta_width(saved_table):
    sizes = [32, 77, 130, 256, 300, 511]
    mats = [torch.from_numpy(workloads.dense_gaussian(n, seed=n + 1)).float().cuda() for n in sizes]
    outs = []
    for bt in (256, 128):
        assert _lib.ld_set_tuning("batched_threads", bt) == 0
        s, l = api.logdet_batched(mats, "f32_plain")
        outs.append((s.clone(), l.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    s1, l1 = api.logdet(mats[3], "f32_plain")
    assert float(outs[1][0][3]) == float(s1) and float(outs[1][1][3]) == float(l1)


def test_ld_tune_blocked_and_batched(tmp_path, monkeypatch, saved_table):
    monkeypatch.setenv("LD_TUNE_CACHE", str(tmp_path))
    t = tune.autotune([3000], "f32_3xtf32")
    assert t["blocked_b"] in (64, 128)
    assert t["blocked_pair_min_n"] in (0, 3001)
    assert t["rankb_2sm"] in (0, 1)
    t = tune.autotune([40, 130, 300, 520], "f32_plain")
    for k in (0, 2, 4, 8):
        assert t[f"batched_kb_{k}"] in (8, 16)
    assert t["batched_threads"] in (128, 256)
    files = os.listdir(tmp_path)
    assert len(files) == 1 and files[0].endswith(".tune")
    # a fresh process with the cache directory set starts from the stored table
    want = tune.table()
    code = ("import json, paper_1811_08057_gb300 as pk; from paper_1811_08057_gb300 import tune; "
            "pk.load(); print(json.dumps(tune.table()))")
    env = dict(os.environ, LD_TUNE_CACHE=str(tmp_path))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    import json
    assert json.loads(out.stdout.strip().splitlines()[-1]) == want


def test_blocked_panel_width_64_parity(saved_table):
    n = 700
    A = workloads.dense_gaussian(n, seed=9, var=1.0 / n) + 2.0 * np.eye(n)
    import oracle
    ref = oracle.logdet(A)
    _lib.ld_set_tuning("blocked_b", 64)
    for pair_min in (1 << 40, 0):
        _lib.ld_set_tuning("blocked_pair_min_n", pair_min)
        for mode in ["f32_3xtf32", "f64_blocked"]:
            s, l = api.logdet(torch.from_numpy(A).cuda(), mode)
            assert float(s) == ref.sign
            tol = 1e-12 if mode == "f64_blocked" else 1e-5
            assert abs(float(l) - ref.logabs) <= tol * max(1.0, abs(ref.logabs))
        Ad, sgn, la, perm = workloads.dyadic_lu(300, seed=1)
        f = api.logdet_factor(torch.from_numpy(Ad).cuda(), "f32_3xtf32")
        assert np.array_equal(f.pivot_labels().cpu().numpy(), perm)


def test_fresh_process_narrow_panels_first():
    """In a fresh process, sweeps with narrow panels first (b = 64, then a matrix
    smaller than one panel) must not cap the shared memory of later full panels;
    ld_tune itself times b = 64 before b = 128."""
    code = (
        "import json, torch, numpy as np; "
        "from paper_1811_08057_gb300 import api, _lib, tune; "
        "assert _lib.ld_set_tuning('blocked_b', 64) == 0; "
        "g = torch.Generator().manual_seed(1); "
        "A = (torch.randn(700, 700, generator=g, dtype=torch.float64) / 700 ** 0.5 + 2 * torch.eye(700, dtype=torch.float64)).cuda(); "
        "s1, l1 = api.logdet(A, 'f32_3xtf32'); "
        "assert _lib.ld_set_tuning('blocked_b', 128) == 0; "
        "s2, l2 = api.logdet(A, 'f32_3xtf32'); "
        "s3, l3 = api.logdet(A[:100, :100].contiguous(), 'f64_blocked'); "
        "s4, l4 = api.logdet(A, 'f64_blocked'); "
        "t = tune.autotune([2000], 'f32_3xtf32'); "
        "print(json.dumps([float(l1), float(l2), float(l3), float(l4), float(s1 * s2 * s3 * s4)]))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    import json
    l1, l2, l3, l4, s = json.loads(out.stdout.strip().splitlines()[-1])
    assert s == 1.0
    assert abs(l1 - l4) <= 1e-5 * max(1.0, abs(l4)) and abs(l2 - l4) <= 1e-5 * max(1.0, abs(l4))


@pytest.mark.parametrize("mode,pair_min", [("f32_3xtf32", 0), ("f32_3xtf32", 10 ** 9),
                                           ("f64_ozaki", 10 ** 9), ("f64_blocked", 10 ** 9)])
def test_one_stream_sweep_same_bits(saved_table, mode, pair_min):
    """sweep_pipeline = 0 runs the blocked sweep on the caller's stream only: the
    same operations per element, so the same bits as the pipelined sweep."""
    n = 1500
    A = torch.from_numpy(workloads.dense_gaussian(n, seed=8, var=1.0 / n)).cuda()
    assert _lib.ld_set_tuning("blocked_pair_min_n", pair_min) == 0
    out = []
    try:
        for pipe in (1, 0):
            assert _lib.ld_set_tuning("sweep_pipeline", pipe) == 0
            f = api.logdet_factor(A, mode)
            torch.cuda.synchronize()
            out.append((float(f.sign), float(f.logabs), f.pivot_labels().clone()))
    finally:
        _lib.ld_set_tuning("sweep_pipeline", 1)
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert torch.equal(out[0][2], out[1][2])
