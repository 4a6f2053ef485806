"""The torch binding refuses host tensors and unknown modes before any device
work: the product path has no CPU fallback (the oracle is test infrastructure)."""
import pytest
import torch

from paper_1811_08057_gb300 import api


def test_logdet_rejects_host_tensor():
    with pytest.raises(ValueError, match="CUDA"):
        api.logdet(torch.eye(4, dtype=torch.float64), "f64_plain")


def test_factor_rejects_host_tensor():
    with pytest.raises(ValueError, match="CUDA"):
        api.logdet_factor(torch.eye(4, dtype=torch.float32), "f32_plain")


def test_unknown_mode_rejected():
    with pytest.raises(ValueError, match="unknown mode"):
        api._mode_code("f16_magic")


def test_batched_rejects_host_tensors():
    with pytest.raises(ValueError, match="CUDA"):
        api.logdet_batched([torch.eye(3), torch.eye(5)], "f32_plain")


def test_autograd_rejects_host_tensor():
    X = torch.eye(4, dtype=torch.float32, requires_grad=True)
    with pytest.raises(ValueError, match="CUDA"):
        api.logabsdet(X, "f32_3xtf32")
