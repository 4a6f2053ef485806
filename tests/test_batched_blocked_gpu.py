"""Batched blocked sweep (ld_logdet_batched[_factor] in the FP32 tensor-core
modes: a batch of one size, panel by panel across the batch).

Each matrix takes the operations of the single-matrix blocked sweep (the same
panel kernel on one CTA instead of a 16-CTA cluster, the same multiplier,
transpose and tensor-core update kernels, the same log-sum order), so results are
compared bit for bit with ld_logdet in the same mode, and with the oracle within
the mode's tolerance.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_1811_08057_gb300 import api, _lib

pytestmark = pytest.mark.gpu

TOL = {"f32_3xtf32": 1e-5, "f32_bf16x3": 1e-4, "f32_tf32": 2e-2}


def rel_err(got, want):
    return abs(got - want) / max(abs(want), 1.0)


@pytest.mark.parametrize("mode", ["f32_3xtf32", "f32_bf16x3", "f32_tf32"])
@pytest.mark.parametrize("n", [1, 2, 100, 128, 129, 300])
def test_batched_blocked_vs_oracle_and_single(mode, n):
    mats = workloads.batched_covariances([n] * 5, seed=20 + n)
    dev = [torch.from_numpy(A).float().cuda() for A in mats]
    s, l = api.logdet_batched(dev, mode)
    s, l = s.cpu().numpy(), l.cpu().numpy()
    for i, A in enumerate(mats):
        ref = oracle.logdet(dev[i].double().cpu().numpy())
        assert s[i] == ref.sign, (i, s[i], ref.sign)
        assert rel_err(l[i], ref.logabs) <= TOL[mode], (mode, n, i, l[i], ref.logabs)
        s1, l1 = api.logdet(dev[i], mode)
        assert float(s1) == s[i] and float(l1) == l[i], (mode, n, i, float(l1), l[i])


def test_batched_blocked_dense_512():
    """Nonsymmetric well-conditioned 512^2 matrices (several panels, pivoting)."""
    n = 512
    mats = [workloads.dense_gaussian(n, seed=60 + i, var=1.0 / n) + 2.0 * np.eye(n)
            for i in range(4)]
    dev = [torch.from_numpy(A).float().cuda() for A in mats]
    s, l = api.logdet_batched(dev, "f32_3xtf32")
    for i in range(4):
        ref = oracle.logdet(dev[i].double().cpu().numpy())
        assert float(s[i]) == ref.sign
        assert rel_err(float(l[i]), ref.logabs) <= 1e-5
        s1, l1 = api.logdet(dev[i], "f32_3xtf32")
        assert float(l1) == float(l[i])


def test_batched_blocked_wrong_size_is_nan():
    n = 64
    mats = workloads.batched_covariances([n, n, 40], seed=9)
    dev = [torch.from_numpy(A).float().cuda() for A in mats]
    batch = api.BatchedInputs(dev)
    signs = torch.empty(3, dtype=torch.float64, device="cuda")
    logabs = torch.empty(3, dtype=torch.float64, device="cuda")
    assert _lib.ld_logdet_batched(batch.ptrs.data_ptr(), batch.dtype_code, batch.n.data_ptr(),
                                  batch.lda.data_ptr(), 3, n, _lib.MODES["f32_3xtf32"], None,
                                  signs.data_ptr(), logabs.data_ptr()) == 0
    l = logabs.cpu().numpy()
    assert math.isfinite(l[0]) and math.isfinite(l[1]) and math.isnan(l[2])


def test_batched_blocked_autograd_vs_fp64_inverse():
    B, n = 4, 300
    mats = [workloads.spd_spectrum(n, seed=40 + i, lo=1e-2, hi=1.0)[0] for i in range(B)]
    X = torch.from_numpy(np.stack(mats)).float().cuda().requires_grad_(True)
    out = api.logabsdet(X, "f32_3xtf32")
    w = torch.linspace(0.5, 1.5, B, device="cuda")
    (out * w).sum().backward()
    for i in range(B):
        R = oracle.grad_logabs(X[i].detach().double().cpu().numpy(), float(w[i]))
        G = X.grad[i].double().cpu().numpy()
        assert np.linalg.norm(G - R) / np.linalg.norm(R) <= 1e-4
        ref = oracle.logdet(X[i].detach().double().cpu().numpy())
        assert rel_err(float(out[i]), ref.logabs) <= 1e-5
