"""Backward G = g * A^{-T} (ld_logdet_backward[_batched], LogAbsDet) against the
FP64 definition (Jacobi's formula via a library inverse), central finite
differences of the FP64 oracle, and torch.autograd.gradcheck.

Tolerances (relative Frobenius norm against the FP64 inverse): FP64 records
1e-10; FP32 records (split-TF32 block products, FP32 substitution) 1e-4 on
well-conditioned matrices.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_1811_08057_gb300 import api, _lib

pytestmark = pytest.mark.gpu


def rel_fro(G, R):
    return float(np.linalg.norm(G - R) / np.linalg.norm(R))


@pytest.mark.parametrize("mode,tol", [("f64_plain", 1e-10), ("f32_plain", 1e-4),
                                      ("f64_blocked", 1e-10), ("f64_ozaki", 1e-10),
                                      ("f32_3xtf32", 1e-4)])
@pytest.mark.parametrize("n", [1, 2, 5, 64, 129, 300])
def test_backward_matches_fp64_inverse(mode, tol, n):
    A = workloads.dense_gaussian(n, seed=500 + n) + 3.0 * np.eye(n)
    f = api.logdet_factor(torch.from_numpy(A).cuda(), mode)
    G = api.logdet_backward(f, 0.75).double().cpu().numpy()
    R = oracle.grad_logabs(A, 0.75)
    assert rel_fro(G, R) <= tol, (mode, n, rel_fro(G, R))


def test_backward_central_differences():
    """<G, E> against central differences of the FP64 oracle log|det| (h = 1e-3)."""
    n = 40
    A = workloads.spd_spectrum(n, seed=4, lo=1e-2, hi=1.0)[0]
    f = api.logdet_factor(torch.from_numpy(A).cuda(), "f64_plain")
    G = api.logdet_backward(f, 1.0).cpu().numpy()
    rng = np.random.default_rng(1)
    h = 1e-3
    for k in range(8):
        if k < 4:
            E = np.zeros((n, n))
            E[rng.integers(n), rng.integers(n)] = 1.0
        else:
            E = rng.standard_normal((n, n))
            E /= np.linalg.norm(E)
        fd = (oracle.logdet(A + h * E).logabs - oracle.logdet(A - h * E).logabs) / (2 * h)
        assert abs(fd - float(np.sum(G * E))) <= 1e-4 * max(1.0, abs(fd))


def test_gradcheck_fp64():
    n = 12
    A = torch.from_numpy(workloads.dense_gaussian(n, seed=3) + 2 * np.eye(n)).cuda()
    A.requires_grad_(True)
    assert torch.autograd.gradcheck(lambda X: api.logabsdet(X, "f64_plain"), (A,), eps=1e-6,
                                    atol=1e-6, rtol=1e-5)


def test_autograd_batched_matches_single():
    B, n = 6, 200
    mats = [workloads.spd_spectrum(n, seed=10 + i, lo=1e-2, hi=1.0)[0] for i in range(B)]
    X = torch.from_numpy(np.stack(mats)).float().cuda().requires_grad_(True)
    out = api.logabsdet(X, "f32_plain")
    w = torch.linspace(0.5, 1.5, B, device="cuda")
    (out * w).sum().backward()
    for i in range(B):
        R = oracle.grad_logabs(X[i].detach().double().cpu().numpy(), float(w[i]))
        assert rel_fro(X.grad[i].double().cpu().numpy(), R) <= 1e-4
        ref = oracle.logdet(X[i].detach().double().cpu().numpy())
        assert abs(float(out[i]) - ref.logabs) <= 1e-5 * max(1.0, abs(ref.logabs))


def test_batched_factor_records_reconstruct():
    sizes = [70, 70, 70]
    mats = [workloads.dense_gaussian(n, seed=n + i) for i, n in enumerate(sizes)]
    X = torch.from_numpy(np.stack(mats)).cuda()
    batch = api.BatchedInputs(list(X))
    buf, offs = api._aligned_records(sizes, _lib.LD_F64_PLAIN, "cuda")
    recs = torch.tensor([buf.data_ptr() + o for o in offs], dtype=torch.int64, device="cuda")
    s = torch.empty(3, dtype=torch.float64, device="cuda")
    l = torch.empty(3, dtype=torch.float64, device="cuda")
    assert _lib.ld_logdet_batched_factor(batch.ptrs.data_ptr(), 0, batch.n.data_ptr(),
                                         batch.lda.data_ptr(), 3, 70, 0, None, recs.data_ptr(),
                                         s.data_ptr(), l.data_ptr()) == 0
    for i, A in enumerate(mats):
        n = sizes[i]
        size = _lib.ld_factors_size(n, 0)
        f = api.parse_factors(buf[offs[i]:offs[i] + size], n, "f64_plain")
        ref = oracle.logdet(A)
        assert np.array_equal(f.pivot_labels().cpu().numpy(), ref.piv_label)
        assert np.array_equal(f.pivval.cpu().numpy(), ref.piv_value)
        F = f.F[:, :n].cpu().numpy()[:, ::-1]
        L = np.tril(F)
        U = np.triu(F, 1) + np.eye(n)
        AQJ = A[:, f.colperm.cpu().numpy()][:, ::-1]
        assert np.abs(L @ U - AQJ).max() <= 1e-12 * n


@pytest.mark.parametrize("mode", ["f32_plain", "f32_3xtf32"])
def test_backward_config_256x1024_sampled(mode):
    """256 SPD 1024^2 (eigenvalues log-uniform in [1e-2, 1]), FP32: batched forward
    (persistent plain sweep, or the batched blocked 3xTF32 sweep) and backward; 4
    sampled gradients against the FP64 inverse."""
    B, n = 256, 1024
    g = torch.Generator(device="cuda").manual_seed(4)
    lam = 10.0 ** (-2.0 * torch.rand(B, n, generator=g, device="cuda", dtype=torch.float64))
    Q, R = torch.linalg.qr(torch.randn(B, n, n, generator=g, device="cuda", dtype=torch.float64))
    Q = Q * torch.sign(torch.diagonal(R, dim1=1, dim2=2))[:, None, :]
    A = (Q * lam[:, None, :]) @ Q.transpose(1, 2)
    A = (0.5 * (A + A.transpose(1, 2))).float()
    del Q, R
    X = A.clone().requires_grad_(True)
    out = api.logabsdet(X, mode)
    out.sum().backward()
    torch.cuda.synchronize()
    exact = torch.log(lam).sum(dim=1)
    assert torch.max(torch.abs(out.double() - exact) / exact.abs().clamp(min=1)).item() <= 1e-4
    for i in [0, 77, 150, 255]:
        Ai = A[i].double().cpu().numpy()
        Rg = oracle.grad_logabs(Ai, 1.0)
        assert rel_fro(X.grad[i].double().cpu().numpy(), Rg) <= 1e-4


def test_config5_central_differences():
    """The 256 x 1024^2 gradient workload (eigenvalues log-uniform in [1e-2, 1],
    FP32, batched blocked 3xTF32 forward and backward): on 4 sampled matrices,
    <G, E> for 16 single entries and 16 random unit-Frobenius directions E against
    central differences of log|det| with h = 1e-3 (Richardson-combined with h/2,
    which removes the h^2 term), the log-determinants taken by the FP64 plain
    sweep (bit-identical to the FP64 oracle's operations) in batched launches."""
    B, n = 256, 1024
    g = torch.Generator(device="cuda").manual_seed(4)
    lam = 10.0 ** (-2.0 * torch.rand(B, n, generator=g, device="cuda", dtype=torch.float64))
    Q, R = torch.linalg.qr(torch.randn(B, n, n, generator=g, device="cuda", dtype=torch.float64))
    Q = Q * torch.sign(torch.diagonal(R, dim1=1, dim2=2))[:, None, :]
    A = (Q * lam[:, None, :]) @ Q.transpose(1, 2)
    A = (0.5 * (A + A.transpose(1, 2))).float()
    del Q, R
    X = A.clone().requires_grad_(True)
    api.logabsdet(X, "f32_3xtf32").sum().backward()
    torch.cuda.synchronize()
    rng = np.random.default_rng(12)
    h = 1e-3
    worst = 0.0
    for i in [0, 85, 170, 255]:
        A64 = A[i].double()
        G = X.grad[i].double()
        dirs = []
        for _ in range(16):
            E = torch.zeros(n, n, dtype=torch.float64, device="cuda")
            r, c = rng.integers(0, n, size=2)
            E[r, c] = 1.0
            dirs.append(E)
        for _ in range(16):
            E = torch.from_numpy(rng.standard_normal((n, n))).cuda()
            dirs.append(E / torch.linalg.norm(E))
        mats = [(A64 + sgn * step * E).contiguous() for E in dirs
                for sgn, step in ((1, h), (-1, h), (1, h / 2), (-1, h / 2))]
        _, la = api.logdet_batched(mats, "f64_plain")
        la = la.cpu().numpy().reshape(len(dirs), 4)
        del mats
        for k, E in enumerate(dirs):
            d1 = (la[k, 0] - la[k, 1]) / (2 * h)
            d2 = (la[k, 2] - la[k, 3]) / h
            fd = (4.0 * d2 - d1) / 3.0
            ip = float((G * E).sum())
            err = abs(fd - ip) / max(abs(fd), 1.0)
            worst = max(worst, err)
            assert err <= 1e-4, (i, k, fd, ip)
    print(f"config 5 central differences: worst relative error {worst:.2e}")
