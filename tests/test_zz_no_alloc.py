"""ld_logdet_noalloc (the entry point for callers that cannot allocate device
memory) agrees with ld_logdet on two calls in a row.

Such callers (a stream capture that forbids allocations, a fixed device-memory
budget, an allocator owned by another framework) get the plain FP64 sweep with a
fixed workspace in the library's device memory. This file is collected last so
that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from paper_1811_08057_gb300 import _lib

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 log|det| tolerance of the other parity tests


def _both(A):
    n = A.shape[0]
    stream = torch.cuda.current_stream().cuda_stream
    ref = torch.empty(2, dtype=torch.float64, device="cuda")
    got = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    assert _lib.ld_logdet(A.data_ptr(), _lib.LD_DTYPE_F64, n, n, _lib.LD_F64_PLAIN, stream,
                          ref.data_ptr(), ref.data_ptr() + 8) == 0
    assert _lib.ld_logdet_noalloc(A.data_ptr(), _lib.LD_DTYPE_F64, n, n, stream, got.data_ptr(),
                                  got.data_ptr() + 8) == 0
    torch.cuda.synchronize()
    return ref.cpu().numpy(), got.cpu().numpy()


def test_noalloc_matches_ld_logdet_two_calls():
    # two calls in a row through the one shared workspace: a larger matrix, then a
    # smaller one (the second must not see the first one's leftovers)
    for n, seed in [(1000, 0), (257, 5)]:
        A = torch.from_numpy(workloads.dense_gaussian(n, seed=seed)).cuda()
        ref, got = _both(A)
        assert got[0] == ref[0]
        assert abs(got[1] - ref[1]) <= TOL * max(1.0, abs(ref[1]))


def test_noalloc_host_outputs_and_limit():
    n = 64
    A = torch.from_numpy(workloads.dense_gaussian(n, seed=9)).cuda()
    ref, _ = _both(A)
    hs, hl = ctypes.c_double(), ctypes.c_double()
    assert _lib.ld_logdet_noalloc(A.data_ptr(), _lib.LD_DTYPE_F64, n, n,
                                  torch.cuda.current_stream().cuda_stream, ctypes.addressof(hs),
                                  ctypes.addressof(hl)) == 0
    assert hs.value == ref[0] and abs(hl.value - ref[1]) <= TOL * max(1.0, abs(ref[1]))
    # above the fixed workspace's bound: rejected before any device work
    assert _lib.ld_logdet_noalloc(A.data_ptr(), _lib.LD_DTYPE_F64, 1025, 1025, None,
                                  ctypes.addressof(hs), ctypes.addressof(hl)) == 2


def test_noalloc_allocates_nothing(monkeypatch):
    """The entry point's promise: with the library's allocator made to fail
    (LD_FAULT_INJECT_ALLOC=1, read by the library at each allocation),
    ld_logdet reports LD_ERR_ALLOC while ld_logdet_noalloc still returns LD_OK and
    the same result as before."""
    n = 300
    A = torch.from_numpy(workloads.dense_gaussian(n, seed=31)).cuda()
    ref, _ = _both(A)
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    monkeypatch.setenv("LD_FAULT_INJECT_ALLOC", "1")
    try:
        assert _lib.ld_logdet(A.data_ptr(), _lib.LD_DTYPE_F64, n, n, _lib.LD_F64_PLAIN, stream,
                              out.data_ptr(), out.data_ptr() + 8) == 3
        assert _lib.ld_logdet_noalloc(A.data_ptr(), _lib.LD_DTYPE_F64, n, n, stream,
                                      out.data_ptr(), out.data_ptr() + 8) == 0
    finally:
        monkeypatch.delenv("LD_FAULT_INJECT_ALLOC")
    got = out.cpu().numpy()
    assert got[0] == ref[0] and abs(got[1] - ref[1]) <= TOL * max(1.0, abs(ref[1]))


def test_noalloc_fp32_input():
    """FP32 input is widened into the FP64 sweep, exactly as ld_logdet does for
    FP32 input in the FP64 plain mode."""
    n = 500
    A = torch.from_numpy(workloads.dense_gaussian(n, seed=12)).float().cuda()
    stream = torch.cuda.current_stream().cuda_stream
    ref = torch.empty(2, dtype=torch.float64, device="cuda")
    got = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    assert _lib.ld_logdet(A.data_ptr(), _lib.LD_DTYPE_F32, n, n, _lib.LD_F64_PLAIN, stream,
                          ref.data_ptr(), ref.data_ptr() + 8) == 0
    for _ in range(2):
        assert _lib.ld_logdet_noalloc(A.data_ptr(), _lib.LD_DTYPE_F32, n, n, stream,
                                      got.data_ptr(), got.data_ptr() + 8) == 0
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert g[0] == r[0]
        assert abs(g[1] - r[1]) <= TOL * max(1.0, abs(r[1]))
