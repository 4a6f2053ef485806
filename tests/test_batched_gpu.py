"""Parity of the batched persistent sweep with the oracle and with single sweeps.

The batched kernel applies each panel's rank-1 updates to a trailing element in
pivot order with one FMA each, i.e. the plain sweep's exact operation sequence, so
in FP64 it must agree bit for bit with ld_logdet in f64_plain mode (same pivots,
same log-sum order), and with the oracle within 1e-12. FP32: 1e-5 relative.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_1811_08057_gb300 import api, _lib

pytestmark = pytest.mark.gpu


def rel_err(got, want):
    return abs(got - want) / max(abs(want), 1.0)


def make_batch(sizes, seed, dtype=torch.float64):
    mats = workloads.batched_covariances(sizes, seed=seed)
    return mats, [torch.from_numpy(A).to(dtype).cuda() for A in mats]


@pytest.mark.parametrize("mode,dtype,tol", [("f64_plain", torch.float64, 1e-12),
                                            ("f32_plain", torch.float32, 1e-5)])
def test_batched_uneven_sizes_vs_oracle(mode, dtype, tol):
    sizes = [1, 2, 17, 32, 33, 48, 100, 160, 255, 256, 257, 300, 512, 3, 64]
    mats, dev = make_batch(sizes, seed=7, dtype=dtype)
    s, l = api.logdet_batched(dev, mode)
    s, l = s.cpu().numpy(), l.cpu().numpy()
    for i, A in enumerate(mats):
        ref = oracle.logdet(dev[i].double().cpu().numpy())
        assert s[i] == ref.sign, i
        assert rel_err(l[i], ref.logabs) <= tol, (i, sizes[i], l[i], ref.logabs)


def test_batched_f64_bitwise_equals_single():
    rng = np.random.default_rng(3)
    sizes = [int(x) for x in rng.integers(1, 400, size=24)]
    mats = [workloads.dense_gaussian(n, seed=100 + n) for n in sizes]
    dev = [torch.from_numpy(A).cuda() for A in mats]
    s, l = api.logdet_batched(dev, "f64_plain")
    for i, A in enumerate(dev):
        ss, ll = api.logdet(A, "f64_plain")
        assert float(s[i]) == float(ss)
        assert float(l[i]) == float(ll), (i, sizes[i])


def test_batched_dyadic_exact():
    cases = [workloads.dyadic_lu(n, seed=n) for n in [5, 16, 17, 64, 200]]
    dev = [torch.from_numpy(c[0]).float().cuda() for c in cases]
    s, l = api.logdet_batched(dev, "f32_plain")
    for i, (A, sgn, logabs, perm) in enumerate(cases):
        assert float(s[i]) == sgn
        assert rel_err(float(l[i]), logabs) < 1e-14


def test_batched_edge_cases():
    A = torch.from_numpy(workloads.dense_gaussian(40, seed=1)).cuda()
    Z = A.clone()
    Z[10] = 0
    N = A.clone()
    N[5, 5] = float("nan")
    E = torch.zeros(0, 0, dtype=torch.float64, device="cuda")
    s, l = api.logdet_batched([A, Z, N, E], "f64_plain")
    ref = oracle.logdet(A.cpu().numpy())
    assert float(s[0]) == ref.sign and rel_err(float(l[0]), ref.logabs) <= 1e-12
    assert float(s[1]) == 0.0 and float(l[1]) == -math.inf
    assert math.isnan(float(s[2])) and math.isnan(float(l[2]))
    assert float(s[3]) == 1.0 and float(l[3]) == 0.0
    # a size above the declared bound gives NaN for that matrix only
    b = api.BatchedInputs([A, A])
    b.n_max = 30
    s, l = api.logdet_batched(b, "f64_plain")
    assert math.isnan(float(s[0])) and math.isnan(float(l[1]))
    # count 0 is a no-op; a bad mode is rejected
    assert _lib.ld_logdet_batched(0, 0, 0, 0, 0, 0, 2, None, 0, 0) == 0
    assert _lib.ld_logdet_batched(0, 0, 0, 0, 1, 8, 9, None, 0, 0) == 1


def test_batched_graph_replay_identical():
    sizes = [64, 128, 32, 200, 96]
    _, dev = make_batch(sizes, seed=11, dtype=torch.float32)
    batch = api.BatchedInputs(dev)
    out = (torch.empty(len(dev), dtype=torch.float64, device="cuda"),
           torch.empty(len(dev), dtype=torch.float64, device="cuda"))
    api.logdet_batched(batch, "f32_plain", out=out)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            api.logdet_batched(batch, "f32_plain", stream=s, out=out)
    g.replay()
    torch.cuda.synchronize()
    first = (out[0].clone(), out[1].clone())
    out[0].zero_()
    out[1].zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(first[0], out[0]) and torch.equal(first[1], out[1])
    direct = api.logdet_batched(batch, "f32_plain")
    assert torch.equal(direct[1], first[1])


def test_batched_config_4096_sampled():
    """4096 covariance matrices, sizes uniform on {32, 48, ..., 512}: 24 sampled
    results against the oracle on the same FP32 values, all results finite."""
    sizes = workloads.batched_sizes(4096, seed=3)
    dev = workloads.batched_covariances_torch(sizes, seed=3, device="cuda")
    s, l = api.logdet_batched(dev, "f32_plain")
    torch.cuda.synchronize()
    assert torch.all(s == 1.0)
    assert torch.all(torch.isfinite(l))
    rng = np.random.default_rng(0)
    for i in rng.choice(4096, size=24, replace=False):
        ref = oracle.logdet(dev[i].double().cpu().numpy())
        assert rel_err(float(l[i]), ref.logabs) <= 1e-5, (i, sizes[i])


def test_batched_f32_bitwise_equals_single():
    """FP32 storage: the batched kernel (column moves from the pivot block, rank-1
    updates per element in pivot order, deferred ordered log-sums) against the
    plain FP32 sweep, bit for bit, with sizes past 512 (three and four columns
    per thread, several trailing-row chunks)."""
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in rng.integers(1, 1000, size=12)] + [513, 768, 999]
    mats = [workloads.dense_gaussian(n, seed=200 + n) for n in sizes]
    dev = [torch.from_numpy(A).float().cuda() for A in mats]
    s, l = api.logdet_batched(dev, "f32_plain")
    for i, A in enumerate(dev):
        ss, ll = api.logdet(A, "f32_plain")
        assert float(s[i]) == float(ss), (i, sizes[i])
        assert float(l[i]) == float(ll), (i, sizes[i], float(l[i]), float(ll))


def test_batched_f32_edge_cases():
    """The deferred FP32 results: all-zero pivot row, NaN, empty matrix and a size
    above the declared bound, each confined to its own matrix."""
    A = torch.from_numpy(workloads.dense_gaussian(40, seed=1)).float().cuda()
    Z = A.clone()
    Z[10] = 0
    N = A.clone()
    N[5, 5] = float("nan")
    E = torch.zeros(0, 0, dtype=torch.float32, device="cuda")
    s, l = api.logdet_batched([A, Z, N, E, A], "f32_plain")
    ss, ll = api.logdet(A, "f32_plain")
    for i in (0, 4):
        assert float(s[i]) == float(ss) and float(l[i]) == float(ll)
    assert float(s[1]) == 0.0 and float(l[1]) == -math.inf
    assert math.isnan(float(s[2])) and math.isnan(float(l[2]))
    assert float(s[3]) == 1.0 and float(l[3]) == 0.0
    b = api.BatchedInputs([A, A[:20, :20].contiguous()])
    b.n_max = 30
    s, l = api.logdet_batched(b, "f32_plain")
    assert math.isnan(float(s[0])) and math.isnan(float(l[0]))
    s2, l2 = api.logdet(A[:20, :20].contiguous(), "f32_plain")
    assert float(s[1]) == float(s2) and float(l[1]) == float(l2)
