"""Other pivot-column rules and column factoring on the plain sweep (ld_logdet_variant).

Sec. 1 names the rules of earlier work (the first nonzero entry, the nonzero
entry closest to 1) and Sec. 2.3 the factoring of the pivot out of its column.
The FP64 plain sweep performs the oracle's operations for every option (one IEEE
divide and one FMA per element, the same FP64 decision), so the pivot labels and
pivot values match the oracle's (same rule and side) bit for bit, on Gaussian
inputs that span several column tiles and a ragged tail. FP32 storage is held to
the FP32 tolerance. The Sec. 2.2 example overflows under closest-to-1 and
first-nonzero and stays finite under max |a_kj|, in FP64 and in FP32.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_1811_08057_gb300 import _lib, api

pytestmark = pytest.mark.gpu

RULES = ["max_abs", "closest_to_one", "first_nonzero"]
SIDES = ["row", "column"]


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("side", SIDES)
@pytest.mark.parametrize("n", [1, 2, 3, 64, 257, 1100])
def test_variant_f64_bitwise_pivots(rule, side, n):
    A = workloads.dense_gaussian(n, seed=400 + n)
    ref = oracle.logdet(A, rule=rule, factor=side)
    f = api.logdet_variant_factor(torch.from_numpy(A).cuda(), "f64_plain", rule, side)
    torch.cuda.synchronize()
    assert np.array_equal(f.pivot_labels().cpu().numpy(), ref.piv_label)
    assert np.array_equal(f.pivval.cpu().numpy(), ref.piv_value)
    assert float(f.sign) == ref.sign
    assert abs(float(f.logabs) - ref.logabs) <= 1e-12 * max(1.0, abs(ref.logabs))
    s, l = api.logdet_variant(torch.from_numpy(A).cuda(), "f64_plain", rule, side)
    assert float(s) == ref.sign and float(l) == float(f.logabs)


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("side", SIDES)
def test_variant_f32_tolerance(rule, side):
    n = 300
    A = workloads.dense_gaussian(n, seed=77, var=1.0 / n) + 2.0 * np.eye(n)
    ref = oracle.logdet(A, rule=rule, factor=side)
    s, l = api.logdet_variant(torch.from_numpy(A).float().cuda(), "f32_plain", rule, side)
    assert float(s) == ref.sign
    assert abs(float(l) - ref.logabs) <= 1e-5 * max(1.0, abs(ref.logabs))


def test_variant_default_is_ld_logdet():
    A = torch.from_numpy(workloads.dense_gaussian(500, seed=3)).cuda()
    for mode in ["f64_plain", "f32_plain", "f32_3xtf32"]:
        s0, l0 = api.logdet(A, mode)
        s1, l1 = api.logdet_variant(A, mode, "max_abs", "row")
        assert float(s0) == float(s1) and float(l0) == float(l1)


@pytest.mark.parametrize("dtype,big", [(torch.float64, 1e300), (torch.float32, 1e30)])
def test_sec22_overflow_example(dtype, big):
    """A pivot row of entries 1e-10 and 2.01 above a row of huge entries: dividing
    by the entry closest to 1 (or the first nonzero one) overflows the next
    matrix; the largest |a_kj| keeps it finite (Sec. 2.2)."""
    A = np.array([[1e-10, 2.01, 2.01], [big, big, -big], [1.0, 2.0, 3.0]])
    At = torch.from_numpy(A).to(dtype).cuda()
    mode = "f64_plain" if dtype == torch.float64 else "f32_plain"
    ref = oracle.logdet(A)
    s, l = api.logdet_variant(At, mode, "max_abs", "row")
    assert float(s) == ref.sign and math.isfinite(float(l))
    assert abs(float(l) - ref.logabs) <= (1e-12 if dtype == torch.float64 else 1e-6) * abs(ref.logabs)
    for rule in ("closest_to_one", "first_nonzero"):
        s, l = api.logdet_variant(At, mode, rule, "row")
        assert not math.isfinite(float(l)), (rule, float(l))


def test_variant_rejections():
    A = torch.from_numpy(workloads.dense_gaussian(64, seed=5)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    args = (A.data_ptr(), _lib.LD_DTYPE_F64, 64, 64)
    # blocked modes: only the paper's rule and side
    assert _lib.ld_logdet_variant(*args, _lib.LD_F32_3XTF32, 1, 0, stream, 0, out.data_ptr(),
                                  out.data_ptr() + 8) == 2
    assert _lib.ld_logdet_variant(*args, _lib.LD_F64_BLOCKED, 0, 1, stream, 0, out.data_ptr(),
                                  out.data_ptr() + 8) == 2
    # unknown rule or side
    assert _lib.ld_logdet_variant(*args, _lib.LD_F64_PLAIN, 3, 0, stream, 0, out.data_ptr(),
                                  out.data_ptr() + 8) == 1
    assert _lib.ld_logdet_variant(*args, _lib.LD_F64_PLAIN, 0, 2, stream, 0, out.data_ptr(),
                                  out.data_ptr() + 8) == 1
    # the backward takes row-factored records only
    f = api.logdet_variant_factor(A, "f64_plain", "max_abs", "column")
    g = torch.ones(1, dtype=torch.float64, device="cuda")
    grad = torch.empty(64, 64, dtype=torch.float64, device="cuda")
    assert _lib.ld_logdet_backward(f.record.data_ptr(), g.data_ptr(), grad.data_ptr(), 64,
                                   stream) == 2
