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
