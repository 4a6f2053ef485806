"""The trailing rank-b update D -= A B^T through the C ABI (ld_rankb_update).

Compared element by element with the same update in FP64 on the host. Bounds,
relative to |D| + |A| |B|^T per element (u = unit roundoff of the input format):
  TF32   inputs carry 10 explicit mantissa bits: a few 2^-10, bound 4e-3;
  3xTF32 the dropped lo*lo term and FP32 accumulation: ~2^-20, bound 5e-6;
  BF16x3 hi and lo carry 8 bits each, lo*lo dropped: ~2^-16, bound 1e-4;
  FP64   K FMAs in FP64: bound 1e-14;
  FP64 sliced (Ozaki): each operand row cut at 2^-47 of its largest entry, the
         slice products exact, one FP64 rounding: per element about
         2^-47 (max|a| / mean|a| + max|b| / mean|b|) ~ 1e-13 for Gaussian rows,
         bound 4e-13.
"""
import numpy as np
import pytest
import torch

from paper_1811_08057_gb300 import _lib

pytestmark = pytest.mark.gpu

MODES = {"f64_blocked": (1, torch.float64, 1e-14), "f64_ozaki": (6, torch.float64, 4e-13),
         "f32_tf32": (3, torch.float32, 4e-3),
         "f32_3xtf32": (4, torch.float32, 5e-6), "f32_bf16x3": (5, torch.float32, 1e-4)}

SHAPES = [(128, 128, 64), (1, 1, 64), (129, 257, 128), (300, 1000, 128), (1000, 300, 256),
          (37, 5, 64), (2048, 2048, 128), (2500, 2100, 128), (2500, 2100, 256)]
# the last two run on CTA pairs (at least two waves of tiles; the second half of
# the last pair row lies past M)
OZAKI_SHAPES = [(3, 70, 1), (200, 129, 33), (130, 65, 200), (64, 64, 300)]  # ragged K, K > 128


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("shape", SHAPES)
def test_rankb_update_matches_fp64(mode, shape):
    code, dt, tol = MODES[mode]
    M, N, K = shape
    g = torch.Generator().manual_seed(M * 7919 + N * 31 + K)
    A = torch.randn(M, K, generator=g, dtype=torch.float64).to(dt)
    B = torch.randn(N, K, generator=g, dtype=torch.float64).to(dt)
    D = torch.randn(M, N, generator=g, dtype=torch.float64).to(dt)
    want = D.double() - A.double() @ B.double().T
    scale = D.double().abs() + A.double().abs() @ B.double().abs().T
    Ad, Bd, Dd = A.cuda(), B.cuda(), D.cuda()
    rc = _lib.ld_rankb_update(code, M, N, K, Ad.data_ptr(), K, Bd.data_ptr(), K, Dd.data_ptr(), N,
                              torch.cuda.current_stream().cuda_stream)
    assert rc == 0, _lib.STATUS.get(rc)
    got = Dd.double().cpu()
    err = ((got - want).abs() / scale).max().item()
    assert err <= tol, f"{mode} {shape}: {err:.3e} > {tol:.1e}"


@pytest.mark.parametrize("pad", [12, 10, 42])
def test_rankb_strided_leading_dims(pad):
    """Leading dimensions larger than the logical widths (views into bigger buffers):
    D rows 16-byte aligned (pad 10, 42) or not (pad 12), with whole and partial
    32 x 32 output blocks."""
    M, N, K = 200, 150, 64
    g = torch.Generator().manual_seed(5 + pad)
    A = torch.randn(M, K + 64, generator=g)
    B = torch.randn(N, K + 128, generator=g)
    D = torch.randn(M, N + pad, generator=g)
    want = D[:, :N].double() - A[:, :K].double() @ B[:, :K].double().T
    Ad, Bd, Dd = A.cuda(), B.cuda(), D.cuda()
    rc = _lib.ld_rankb_update(4, M, N, K, Ad.data_ptr(), K + 64, Bd.data_ptr(), K + 128,
                              Dd.data_ptr(), N + pad, torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    got = Dd.cpu()
    assert torch.equal(got[:, N:], D[:, N:]), "columns beyond N were touched"
    scale = D[:, :N].double().abs() + A[:, :K].double().abs() @ B[:, :K].double().abs().T
    assert ((got[:, :N].double() - want).abs() / scale).max().item() <= 5e-6


def test_rankb_rejects_bad_k():
    A = torch.zeros(8, 40, device="cuda")
    assert _lib.ld_rankb_update(4, 8, 8, 40, A.data_ptr(), 40, A.data_ptr(), 40, A.data_ptr(), 40,
                                None) == 2
    assert _lib.ld_rankb_update(0, 8, 8, 64, A.data_ptr(), 64, A.data_ptr(), 64, A.data_ptr(), 64,
                                None) == 1


def test_bf16x3_error_is_the_split():
    """Where BF16x3's error comes from. Inputs already representable in BF16 split
    exactly (lo = 0), so only the tensor cores' FP32 accumulation is left: the
    error, relative to |A| |B|^T, is at the FP32 level. General FP32 inputs lose
    the bits past the two 8-bit pieces (up to 2^-16 per product): an error more
    than ten times larger, at the size that split predicts (about
    0.3 * 2^-16 * sqrt(3) per product, 1 / sqrt(K) after the sum of K products
    of random sign)."""
    M = N = 1024
    K = 128
    g = torch.Generator().manual_seed(77)
    A = torch.randn(M, K, generator=g)
    B = torch.randn(N, K, generator=g)

    def rms_err(A, B):
        D = torch.zeros(M, N, device="cuda")
        Ad, Bd = A.cuda(), B.cuda()
        assert _lib.ld_rankb_update(5, M, N, K, Ad.data_ptr(), K, Bd.data_ptr(), K,
                                    D.data_ptr(), N, torch.cuda.current_stream().cuda_stream) == 0
        want = -(A.double() @ B.double().T)
        scale = A.double().abs() @ B.double().abs().T
        return ((D.double().cpu() - want) / scale).pow(2).mean().sqrt().item()

    exact = rms_err(A.bfloat16().float(), B.bfloat16().float())
    general = rms_err(A, B)
    predicted = 0.3 * 2.0 ** -16 * 3 ** 0.5 / K ** 0.5
    print(f"BF16x3 rms error: split-exact inputs {exact:.2e}, general {general:.2e} "
          f"(split estimate {predicted:.2e})")
    assert exact <= 5e-8
    assert general >= 10 * exact
    assert 0.3 * predicted <= general <= 3 * predicted


@pytest.mark.parametrize("shape", OZAKI_SHAPES)
def test_ozaki_any_k(shape):
    """The sliced FP64 update takes any K (zero-padded chunks of 32, passes of 128)."""
    M, N, K = shape
    g = torch.Generator().manual_seed(K + 17)
    A = torch.randn(M, K, generator=g, dtype=torch.float64)
    B = torch.randn(N, K, generator=g, dtype=torch.float64)
    D = torch.randn(M, N, generator=g, dtype=torch.float64)
    want = D - A @ B.T
    scale = D.abs() + A.abs() @ B.abs().T
    Ad, Bd, Dd = A.cuda(), B.cuda(), D.cuda()  # held: the call only sees raw pointers
    rc = _lib.ld_rankb_update(6, M, N, K, Ad.data_ptr(), K, Bd.data_ptr(), K,
                              Dd.data_ptr(), N, torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    assert ((Dd.cpu() - want).abs() / scale).max().item() <= 4e-13


def test_ozaki_exact_on_small_integers():
    """Integers below 2^7 in magnitude are one slice each and every product and sum
    is exact: the result equals the FP64 one bit for bit, whatever the row scales
    (each row multiplied by its own power of two)."""
    M, N, K = 300, 200, 128
    g = torch.Generator().manual_seed(3)
    sa = torch.pow(2.0, torch.randint(-20, 20, (M, 1), generator=g).double())
    sb = torch.pow(2.0, torch.randint(-20, 20, (N, 1), generator=g).double())
    A = torch.randint(-127, 128, (M, K), generator=g).double() * sa
    B = torch.randint(-127, 128, (N, K), generator=g).double() * sb
    D = torch.randint(-1000, 1000, (M, N), generator=g).double() * (sa @ sb.T)
    # exact on the host too: element (i, j) is an integer below 2^22 times sa_i sb_j
    want = D - A @ B.T
    Ad, Bd, Dd = A.cuda(), B.cuda(), D.cuda()  # held: the call only sees raw pointers
    rc = _lib.ld_rankb_update(6, M, N, K, Ad.data_ptr(), K, Bd.data_ptr(), K,
                              Dd.data_ptr(), N, None)
    assert rc == 0
    assert torch.equal(Dd.cpu(), want)


def test_ozaki_zero_rows_and_nan():
    M, N, K = 130, 70, 64
    g = torch.Generator().manual_seed(9)
    A = torch.randn(M, K, generator=g, dtype=torch.float64)
    B = torch.randn(N, K, generator=g, dtype=torch.float64)
    A[5] = 0.0  # a zero multiplier row leaves its D row unchanged
    A[7, 3] = float("nan")  # a NaN reaches its D row only
    D = torch.randn(M, N, generator=g, dtype=torch.float64)
    Ad, Bd, Dd = A.cuda(), B.cuda(), D.cuda()  # held: the call only sees raw pointers
    rc = _lib.ld_rankb_update(6, M, N, K, Ad.data_ptr(), K, Bd.data_ptr(), K,
                              Dd.data_ptr(), N, None)
    assert rc == 0
    got = Dd.cpu()
    assert torch.equal(got[5], D[5])
    assert torch.isnan(got[7]).all()
    others = [i for i in range(M) if i != 7]
    assert torch.isfinite(got[others]).all()


@pytest.mark.parametrize("mode", ["f32_3xtf32", "f32_bf16x3", "f32_tf32"])
@pytest.mark.parametrize("K", [128, 256])
def test_cta_pairs_match_single_ctas(mode, K):
    """The CTA-pair form (256 x 128 tiles on two SMs) against single CTAs: the same
    products per element, so the results agree to the FP32 rounding of the
    accumulation (compared exactly first, then within a few FP32 ulps of the
    scale), including a last tile row of the pair that lies past M."""
    code, _, tol = MODES[mode]
    M, N = 2500, 2100  # 10 pair rows, the last half past M
    g = torch.Generator().manual_seed(K)
    A = torch.randn(M, K, generator=g).cuda()
    B = torch.randn(N, K, generator=g).cuda()
    D0 = torch.randn(M, N, generator=g).cuda()
    out = []
    old = _lib.ld_get_tuning("rankb_2sm")
    try:
        for two in (0, 1):
            assert _lib.ld_set_tuning("rankb_2sm", two) == 0
            D = D0.clone()
            rc = _lib.ld_rankb_update(code, M, N, K, A.data_ptr(), K, B.data_ptr(), K, D.data_ptr(),
                                      N, torch.cuda.current_stream().cuda_stream)
            assert rc == 0
            out.append(D)
    finally:
        _lib.ld_set_tuning("rankb_2sm", old)
    same = torch.equal(out[0], out[1])
    print(f"{mode} K={K}: bitwise equal {same}")
    scale = (D0.double().abs() + A.double().abs() @ B.double().abs().T)
    assert ((out[0].double() - out[1].double()).abs() / scale).max().item() <= 1e-6
    want = D0.double() - A.double() @ B.double().T
    assert ((out[1].double() - want).abs() / scale).max().item() <= tol
