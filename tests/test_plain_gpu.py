"""Parity of the plain CUDA sweep (FP64 and FP32 rank-1) with the CPU oracle.

FP64 plain: the kernels perform the same IEEE divide and the same single FMA per
minor as the oracle, so the pivot sequence (labels and values) is compared bit for
bit, the sign exactly and log|det| within 1e-12 relative (only the log and the
summation order differ). FP32 plain: sign exact, log|det| within 1e-5 relative;
pivot labels exact on matrices whose sweep is exact in FP32.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_1811_08057_gb300 import _lib, api

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


def rel_err(got, want):
    return abs(got - want) / max(abs(want), 1.0)


def gpu_logdet(A_np, mode, dtype=torch.float64):
    A = torch.from_numpy(np.ascontiguousarray(A_np)).to(dtype).cuda()
    f = api.logdet_factor(A, mode)
    torch.cuda.synchronize()
    return f


def assert_bitexact_f64(A_np, f=None):
    f = f or gpu_logdet(A_np, "f64_plain")
    ref = oracle.logdet(A_np)
    n = A_np.shape[0]
    labels = f.pivot_labels().cpu().numpy()
    pivval = f.pivval.cpu().numpy()
    assert np.array_equal(labels, ref.piv_label), "pivot labels differ"
    assert np.array_equal(pivval, ref.piv_value), "pivot values differ"
    assert float(f.sign) == ref.sign
    assert rel_err(float(f.logabs), ref.logabs) <= F64_TOL
    return f, ref


@pytest.mark.parametrize("n", list(range(1, 65)))
def test_f64_every_small_n(n):
    A = workloads.dense_gaussian(n, seed=1000 + n)
    assert_bitexact_f64(A)


@pytest.mark.parametrize("n", [511, 512, 513, 1023, 1025, 1537])
def test_f64_ragged_tiles(n):
    A = workloads.dense_gaussian(n, seed=n, var=1.0 / n)
    assert_bitexact_f64(A)


def test_f64_config_1000():
    """N = 1000, iid N(0,1), seed 0: full pivot sequence bit for bit."""
    A = workloads.dense_gaussian(1000, seed=0)
    assert_bitexact_f64(A)


@pytest.mark.parametrize("n", [7, 40, 200])
def test_f64_integer_ties(n):
    """Small integers give many equal |a_kj|: the tie-break must match exactly."""
    rng = np.random.default_rng(n)
    A = rng.integers(-3, 4, size=(n, n)).astype(np.float64)
    f = gpu_logdet(A, "f64_plain")
    ref = oracle.logdet(A)
    if ref.sign == 0:
        assert float(f.sign) == 0.0
        return
    assert np.array_equal(f.pivot_labels().cpu().numpy(), ref.piv_label)
    assert np.array_equal(f.pivval.cpu().numpy(), ref.piv_value)


@pytest.mark.parametrize("mode", ["f64_plain", "f32_plain"])
@pytest.mark.parametrize("n", [1, 5, 33, 130, 700])
def test_dyadic_exact_pivots(mode, n):
    """Matrices whose whole sweep is exact in FP32: labels, sign and log|det| exact."""
    A, sgn, logabs, perm = workloads.dyadic_lu(n, seed=n)
    f = gpu_logdet(A, mode, torch.float64)
    assert np.array_equal(f.pivot_labels().cpu().numpy(), perm)
    assert float(f.sign) == sgn
    assert rel_err(float(f.logabs), logabs) < 1e-14


@pytest.mark.parametrize("n", [3, 64, 300, 1000])
def test_f32_plain_tolerance(n):
    A = workloads.dense_gaussian(n, seed=77 + n)
    ref = oracle.logdet(A)
    At = torch.from_numpy(A).cuda()
    s, l = api.logdet(At, "f32_plain")
    assert float(s) == ref.sign
    assert rel_err(float(l), ref.logabs) <= F32_TOL


def test_f32_input_dtype_and_odd_lda():
    n = 301
    A = workloads.dense_gaussian(n, seed=5)
    big = torch.zeros(n, n + 3, dtype=torch.float64, device="cuda")
    big[:, :n] = torch.from_numpy(A).cuda()
    view = big[:, :n]  # lda = n + 3
    assert view.stride(0) == n + 3
    f, ref = assert_bitexact_f64(A, api.logdet_factor(view, "f64_plain"))
    # FP32 input into the FP64 sweep: the oracle sees the same FP32-rounded values
    A32 = torch.from_numpy(A).float().cuda()
    f32in = api.logdet_factor(A32, "f64_plain")
    ref32 = oracle.logdet(A32.double().cpu().numpy())
    assert np.array_equal(f32in.pivval.cpu().numpy(), ref32.piv_value)


def test_unaligned_start():
    n = 97
    A = workloads.dense_gaussian(n, seed=6)
    flat = torch.zeros(n * n + 1, dtype=torch.float64, device="cuda")
    flat[1:] = torch.from_numpy(A).reshape(-1).cuda()
    view = flat[1:].view(n, n)  # starts 8 bytes past a 16-byte boundary
    assert view.data_ptr() % 16 == 8
    assert_bitexact_f64(A, api.logdet_factor(view, "f64_plain"))


@pytest.mark.parametrize("mode", ["f64_plain", "f32_plain"])
def test_conventions(mode):
    # n = 0
    s, l = api.logdet(torch.zeros(0, 0, dtype=torch.float64, device="cuda"), mode)
    assert (float(s), float(l)) == (1.0, 0.0)
    A = workloads.dense_gaussian(40, seed=8)
    Z = A.copy()
    Z[13] = 0.0
    s, l = api.logdet(torch.from_numpy(Z).cuda(), mode)
    assert float(s) == 0.0 and float(l) == -math.inf
    Z = A.copy()
    Z[:, 7] = 0.0
    s, l = api.logdet(torch.from_numpy(Z).cuda(), mode)
    assert float(s) == 0.0 and float(l) == -math.inf
    N = A.copy()
    N[22, 3] = np.nan
    s, l = api.logdet(torch.from_numpy(N).cuda(), mode)
    assert math.isnan(float(s)) and math.isnan(float(l))


def test_host_and_device_outputs():
    import ctypes
    n = 50
    A = workloads.dense_gaussian(n, seed=9)
    At = torch.from_numpy(A).cuda()
    ref = oracle.logdet(A)
    hs, hl = ctypes.c_double(), ctypes.c_double()
    code = _lib.ld_logdet(At.data_ptr(), 0, n, n, 0, torch.cuda.current_stream().cuda_stream,
                          ctypes.addressof(hs), ctypes.addressof(hl))
    assert code == 0
    assert hs.value == ref.sign and rel_err(hl.value, ref.logabs) <= F64_TOL
    # mixed: sign on the device, logabs on the host
    ds = torch.zeros(1, dtype=torch.float64, device="cuda")
    code = _lib.ld_logdet(At.data_ptr(), 0, n, n, 0, torch.cuda.current_stream().cuda_stream,
                          ds.data_ptr(), ctypes.addressof(hl))
    assert code == 0
    assert float(ds[0]) == ref.sign and rel_err(hl.value, ref.logabs) <= F64_TOL


def test_side_stream():
    n = 120
    A = workloads.dense_gaussian(n, seed=10)
    ref = oracle.logdet(A)
    s = torch.cuda.Stream()
    At = torch.from_numpy(A).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        sg, la = api.logdet(At, "f64_plain", stream=s)
    s.synchronize()
    assert float(sg) == ref.sign and rel_err(float(la), ref.logabs) <= F64_TOL


def test_injected_alloc_failure(monkeypatch):
    monkeypatch.setenv("LD_FAULT_INJECT_ALLOC", "1")
    A = torch.eye(8, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.LogdetError) as e:
        api.logdet(A)
    assert e.value.code == 3
    monkeypatch.setenv("LD_FAULT_INJECT_ALLOC", "0")
    s, l = api.logdet(A)
    assert float(s) == 1.0 and float(l) == 0.0


def test_factors_reconstruct_matrix():
    """A Q J = L U from the record (packed Crout factors, reversed column order)."""
    n = 60
    A = workloads.dense_gaussian(n, seed=11)
    f = gpu_logdet(A, "f64_plain")
    F = f.F[:, :n].cpu().numpy()
    FJ = F[:, ::-1]
    L = np.tril(FJ)
    U = np.triu(FJ, 1) + np.eye(n)
    cp = f.colperm.cpu().numpy()
    AQJ = A[:, cp][:, ::-1]
    assert np.allclose(L @ U, AQJ, rtol=0, atol=1e-12 * np.abs(A).max() * n)


def test_f64_config_8000_full_sequence():
    """N = 8000, iid N(0, 1/N), seed 1 (the benchmark's matrix): the oracle runs
    threaded on the host; the whole pivot sequence must match bit for bit."""
    import os
    A = workloads.dense_gaussian(8000, seed=1, var=1.0 / 8000)
    At = torch.from_numpy(A).cuda()
    f = api.logdet_factor(At, "f64_plain")
    torch.cuda.synchronize()
    ref = oracle.logdet(A, nthreads=max(1, (os.cpu_count() or 2)))
    assert np.array_equal(f.pivot_labels().cpu().numpy(), ref.piv_label)
    assert np.array_equal(f.pivval.cpu().numpy(), ref.piv_value)
    assert float(f.sign) == ref.sign
    assert rel_err(float(f.logabs), ref.logabs) <= F64_TOL


def test_wait_limit_runs_out_and_context_stays_usable(monkeypatch):
    """A bounded device wait that runs out: with the grid panel's wait limit at 0
    (the grid-wide panel, selected here with LD_PANEL=grid, polls global-memory
    tags), the tag barrier gives up, the sweep is flagged, the results are NaN and
    the call reports LD_ERR_TIMEOUT. The context stays usable: with the limit
    restored the same call succeeds."""
    import ctypes
    monkeypatch.setenv("LD_PANEL", "grid")
    n = 1000  # 16 panel CTAs and 1000 tag barriers: some wait outlasts a timer tick
    A = workloads.dense_gaussian(n, seed=61)
    At = torch.from_numpy(A).cuda()
    ref = oracle.logdet(A)
    old = _lib.ld_get_tuning("wait_limit_ns")
    assert old == 1_000_000_000
    hs, hl = ctypes.c_double(), ctypes.c_double()
    stream = torch.cuda.current_stream().cuda_stream
    try:
        assert _lib.ld_set_tuning("wait_limit_ns", 0) == 0
        code = _lib.ld_logdet(At.data_ptr(), _lib.LD_DTYPE_F64, n, n, _lib.LD_F64_BLOCKED, stream,
                              ctypes.addressof(hs), ctypes.addressof(hl))
        assert code == 5, _lib.STATUS.get(code)
        assert math.isnan(hs.value) and math.isnan(hl.value)
    finally:
        assert _lib.ld_set_tuning("wait_limit_ns", old) == 0
    code = _lib.ld_logdet(At.data_ptr(), _lib.LD_DTYPE_F64, n, n, _lib.LD_F64_BLOCKED, stream,
                          ctypes.addressof(hs), ctypes.addressof(hl))
    assert code == 0 and hs.value == ref.sign
    assert abs(hl.value - ref.logabs) <= 1e-12 * max(1.0, abs(ref.logabs))
