"""The sharded batched call on one GPU (world size 1, no process group): its
default per-rank work is one ld_logdet_batched call, and the combined vectors
equal a direct batched call bit for bit."""
import pytest
import torch

import workloads
from paper_1811_08057_gb300 import api
from paper_1811_08057_gb300 import dist as ld_dist

pytestmark = pytest.mark.gpu


def test_sharded_batch_single_rank_equals_batched_call():
    sizes = [int(x) for x in workloads.batched_sizes(200, seed=12)]
    mats = workloads.batched_covariances_torch(sizes, seed=12, device="cuda")
    s, l = ld_dist.logdet_batched_distributed(sizes, lambda i: mats[i], "f32_plain", device="cuda")
    s0, l0 = api.logdet_batched(api.BatchedInputs(mats), "f32_plain")
    assert torch.equal(s, s0) and torch.equal(l, l0)
