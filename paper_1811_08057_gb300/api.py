"""Torch-facing wrappers of the C ABI (marshalling only: no arithmetic here)."""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import _lib


def _mode_code(mode) -> int:
    if isinstance(mode, str):
        if mode not in _lib.MODES:
            raise ValueError(f"unknown mode {mode!r}; one of {sorted(_lib.MODES)}")
        return _lib.MODES[mode]
    return int(mode)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return _lib.LD_DTYPE_F64
    if t.dtype == torch.float32:
        return _lib.LD_DTYPE_F32
    raise TypeError(f"unsupported dtype {t.dtype}; float64 or float32")


def _stream_handle(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _check_matrix(A: torch.Tensor):
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square")
    if A.shape[0] > 0 and A.stride(1) != 1:
        raise ValueError("A must be row-major (unit stride along rows)")


def logdet(A: torch.Tensor, mode="f64_plain", stream=None):
    """(sign, log|det A|) as 0-d FP64 CUDA tensors (no host synchronisation).

    mode "f32_tf32" is approximate: its trailing update keeps 10 mantissa bits,
    and on an ill-conditioned matrix even the sign can come out wrong.
    """
    _check_matrix(A)
    n = A.shape[0]
    lda = max(A.stride(0), 1) if n > 0 else 1
    out = torch.empty(2, dtype=torch.float64, device=A.device)
    code = _lib.ld_logdet(A.data_ptr(), _dtype_code(A), n, lda, _mode_code(mode),
                          _stream_handle(stream), out.data_ptr(), out.data_ptr() + 8)
    _lib.check("ld_logdet", code)
    return out[0], out[1]


def logdet_variant(A: torch.Tensor, mode="f64_plain", rule="max_abs", factor="row",
                   stream=None):
    """(sign, log|det A|) with another pivot-column rule ("max_abs", the paper's;
    "closest_to_one" or "first_nonzero", earlier work) or the pivot factored out
    of the "column" instead of the "row"; plain modes only for anything but the
    paper's choices."""
    _check_matrix(A)
    if rule not in _lib.PIVOT_RULES or factor not in _lib.FACTOR_SIDES:
        raise ValueError(f"unknown rule {rule!r} or factor side {factor!r}")
    n = A.shape[0]
    lda = max(A.stride(0), 1) if n > 0 else 1
    out = torch.empty(2, dtype=torch.float64, device=A.device)
    code = _lib.ld_logdet_variant(A.data_ptr(), _dtype_code(A), n, lda, _mode_code(mode),
                                  _lib.PIVOT_RULES[rule], _lib.FACTOR_SIDES[factor],
                                  _stream_handle(stream), 0, out.data_ptr(), out.data_ptr() + 8)
    _lib.check("ld_logdet_variant", code)
    return out[0], out[1]


def logdet_variant_factor(A: torch.Tensor, mode="f64_plain", rule="max_abs", factor="row",
                          stream=None) -> Factors:
    """As logdet_variant, and keeps the factor record (its pivot sequence under the
    chosen rule; with factor="column" F holds the column-factored form)."""
    _check_matrix(A)
    if rule not in _lib.PIVOT_RULES or factor not in _lib.FACTOR_SIDES:
        raise ValueError(f"unknown rule {rule!r} or factor side {factor!r}")
    n = A.shape[0]
    lda = max(A.stride(0), 1) if n > 0 else 1
    mode = _mode_code(mode)
    size = _lib.ld_factors_size(n, mode)
    record = torch.empty(size + 256, dtype=torch.uint8, device=A.device)
    shift = (-record.data_ptr()) % 256
    record = record[shift:shift + size]
    out = torch.empty(2, dtype=torch.float64, device=A.device)
    code = _lib.ld_logdet_variant(A.data_ptr(), _dtype_code(A), n, lda, mode,
                                  _lib.PIVOT_RULES[rule], _lib.FACTOR_SIDES[factor],
                                  _stream_handle(stream), record.data_ptr(), out.data_ptr(),
                                  out.data_ptr() + 8)
    _lib.check("ld_logdet_variant", code)
    return parse_factors(record, n, mode)


@dataclass
class Factors:
    """A factor record (see ld_factors_size in include/logdet.h) and its views."""
    record: torch.Tensor  # uint8, the whole record
    n: int
    mode: int
    F: torch.Tensor       # n x ldf
    colperm: torch.Tensor
    pivpos: torch.Tensor
    pivval: torch.Tensor
    sign: torch.Tensor
    logabs: torch.Tensor

    def pivot_labels(self) -> torch.Tensor:
        """Original column label of the pivot of each step: the column that step s
        eliminates ends at position n-1-s."""
        return torch.flip(self.colperm.long(), dims=[0])


def _align(x, a=256):
    return (x + a - 1) // a * a


def parse_factors(record: torch.Tensor, n: int, mode) -> Factors:
    mode = _mode_code(mode)
    f64 = mode in _lib.F64_MODES
    es = 8 if f64 else 4
    ldf = _align(max(n, 1), 32)
    off = 256
    F = record[off:off + n * ldf * es].view(torch.float64 if f64 else torch.float32)
    F = F.view(n, ldf) if n > 0 else F.view(0, ldf)
    off += _align(n * ldf * es)
    colperm = record[off:off + 4 * n].view(torch.int32)
    off += _align(4 * n)
    pivpos = record[off:off + 4 * n].view(torch.int32)
    off += _align(4 * n)
    pivval = record[off:off + 8 * n].view(torch.float64)
    hdr = record[:256]
    sign = hdr[24:32].view(torch.float64)[0]
    logabs = hdr[32:40].view(torch.float64)[0]
    return Factors(record, n, mode, F, colperm, pivpos, pivval, sign, logabs)


def logdet_factor(A: torch.Tensor, mode="f64_plain", stream=None) -> Factors:
    """Sweep A and keep the factors (packed Crout LU in the swap-to-boundary layout)."""
    _check_matrix(A)
    n = A.shape[0]
    lda = max(A.stride(0), 1) if n > 0 else 1
    mode = _mode_code(mode)
    size = _lib.ld_factors_size(n, mode)
    if size == 0:
        raise ValueError("invalid size or mode")
    record = torch.empty(size + 256, dtype=torch.uint8, device=A.device)
    shift = (-record.data_ptr()) % 256
    record = record[shift:shift + size]
    out = torch.empty(2, dtype=torch.float64, device=A.device)
    code = _lib.ld_logdet_factor(A.data_ptr(), _dtype_code(A), n, lda, mode,
                                 _stream_handle(stream), record.data_ptr(), out.data_ptr(),
                                 out.data_ptr() + 8)
    _lib.check("ld_logdet_factor", code)
    return parse_factors(record, n, mode)


class BatchedInputs:
    """Device arrays (pointers, sizes, leading dimensions) for ld_logdet_batched.

    Keeps references to the matrices so their memory outlives the arrays. Build it
    once and reuse it across calls (or CUDA-graph replays).
    """

    def __init__(self, mats, device=None):
        if len(mats) == 0:
            raise ValueError("empty batch")
        dt = mats[0].dtype
        for A in mats:
            _check_matrix(A)
            if A.dtype != dt:
                raise TypeError("all matrices must share one dtype")
        device = device or mats[0].device
        self.mats = list(mats)
        self.dtype_code = _dtype_code(mats[0])
        self.count = len(mats)
        self.n_max = max(A.shape[0] for A in mats)
        self.ptrs = torch.tensor([A.data_ptr() for A in mats], dtype=torch.int64, device=device)
        self.n = torch.tensor([A.shape[0] for A in mats], dtype=torch.int64, device=device)
        self.lda = torch.tensor([max(A.stride(0), 1) if A.shape[0] else 1 for A in mats],
                                dtype=torch.int64, device=device)


def logdet_batched(batch, mode="f32_plain", stream=None, out=None):
    """sign and log|det| of every matrix of a batch (list of CUDA tensors or a
    BatchedInputs). f64_plain / f32_plain: one persistent launch, any sizes; the
    FP32 tensor-core modes: a batch of one size, blocked panel by panel across the
    batch. Returns (signs, logabs) FP64 tensors."""
    if not isinstance(batch, BatchedInputs):
        batch = BatchedInputs(batch)
    if out is None:
        signs = torch.empty(batch.count, dtype=torch.float64, device=batch.ptrs.device)
        logabs = torch.empty(batch.count, dtype=torch.float64, device=batch.ptrs.device)
    else:
        signs, logabs = out
    code = _lib.ld_logdet_batched(batch.ptrs.data_ptr(), batch.dtype_code, batch.n.data_ptr(),
                                  batch.lda.data_ptr(), batch.count, batch.n_max,
                                  _mode_code(mode), _stream_handle(stream), signs.data_ptr(),
                                  logabs.data_ptr())
    _lib.check("ld_logdet_batched", code)
    return signs, logabs


def _aligned_records(sizes, mode, device):
    """One contiguous buffer holding a 256-B aligned factor record per size."""
    offs, total = [], 0
    for n in sizes:
        total = _align(total)
        offs.append(total)
        total += _lib.ld_factors_size(int(n), mode)
    buf = torch.empty(total + 256, dtype=torch.uint8, device=device)
    shift = (-buf.data_ptr()) % 256
    buf = buf[shift:shift + total]
    return buf, offs


def logdet_backward(f: Factors, g=1.0, stream=None) -> torch.Tensor:
    """G = g * A^{-T} from a factor record (ld_logdet_backward)."""
    dev = f.record.device
    gt = torch.as_tensor(g, dtype=torch.float64, device=dev).reshape(1).contiguous()
    dt = torch.float64 if f.mode in _lib.F64_MODES else torch.float32
    G = torch.empty(f.n, f.n, dtype=dt, device=dev)
    code = _lib.ld_logdet_backward(f.record.data_ptr(), gt.data_ptr(), G.data_ptr(), max(f.n, 1),
                                   _stream_handle(stream))
    _lib.check("ld_logdet_backward", code)
    return G


class LogAbsDet(torch.autograd.Function):
    """log|det A| with gradient g * A^{-T}, both through liblogdet.

    Single matrix (n x n) or a batch (B x n x n, one size). Forward keeps the
    factor records (ld_logdet_factor, or ld_logdet_batched_factor for a batch);
    backward runs ld_logdet_backward_batched on them.
    """

    @staticmethod
    def forward(ctx, A, mode="f32_plain"):
        mode_c = _mode_code(mode)
        batched = A.dim() == 3
        mats = list(A) if batched else [A]
        n = A.shape[-1]
        dev = A.device
        if batched:
            if mode_c in (_lib.LD_F64_BLOCKED, _lib.LD_F64_OZAKI):
                raise ValueError("batched forward supports f64_plain, f32_plain and the FP32 "
                                 "tensor-core modes")
            mats = [M.contiguous() for M in mats]
            batch = BatchedInputs(mats)
            buf, offs = _aligned_records([n] * len(mats), mode_c, dev)
            recs = torch.tensor([buf.data_ptr() + o for o in offs], dtype=torch.int64, device=dev)
            signs = torch.empty(len(mats), dtype=torch.float64, device=dev)
            logabs = torch.empty(len(mats), dtype=torch.float64, device=dev)
            code = _lib.ld_logdet_batched_factor(batch.ptrs.data_ptr(), batch.dtype_code,
                                                 batch.n.data_ptr(), batch.lda.data_ptr(),
                                                 batch.count, batch.n_max, mode_c,
                                                 _stream_handle(None), recs.data_ptr(),
                                                 signs.data_ptr(), logabs.data_ptr())
            _lib.check("ld_logdet_batched_factor", code)
            ctx.keep = (buf, recs, batch)
            out = logabs
        else:
            f = logdet_factor(A.contiguous(), mode_c)
            recs = torch.tensor([f.record.data_ptr()], dtype=torch.int64, device=dev)
            ctx.keep = (f.record, recs, None)
            out = f.logabs.reshape(())
        ctx.meta = (batched, n, mode_c, A.dtype, len(mats))
        return out.to(A.dtype) if A.dtype == torch.float32 else out.clone()

    @staticmethod
    def backward(ctx, grad_out):
        batched, n, mode_c, dtype, count = ctx.meta
        _, recs, _ = ctx.keep
        dev = grad_out.device
        g = grad_out.detach().to(torch.float64).reshape(count).contiguous()
        sdt = torch.float64 if mode_c in _lib.F64_MODES else torch.float32
        G = torch.empty(count, n, n, dtype=sdt, device=dev)
        gptrs = torch.tensor([G[i].data_ptr() for i in range(count)], dtype=torch.int64,
                             device=dev)
        code = _lib.ld_logdet_backward_batched(recs.data_ptr(), count, n, mode_c, g.data_ptr(),
                                               gptrs.data_ptr(), n, _stream_handle(None))
        _lib.check("ld_logdet_backward_batched", code)
        G = G.to(dtype)
        return (G if batched else G[0]), None


def logabsdet(A: torch.Tensor, mode="f32_plain") -> torch.Tensor:
    """Differentiable log|det A| (n x n or B x n x n) through liblogdet."""
    return LogAbsDet.apply(A, mode)


def _csr_arrays(row_ptr: torch.Tensor, col_idx: torch.Tensor):
    if row_ptr.dtype != torch.int64 or col_idx.dtype != torch.int64:
        raise TypeError("row_ptr and col_idx must be int64 tensors")
    if row_ptr.dim() != 1 or col_idx.dim() != 1:
        raise ValueError("row_ptr and col_idx must be 1-D")
    return row_ptr.contiguous(), col_idx.contiguous()


def logdet_sparse(row_ptr: torch.Tensor, col_idx: torch.Tensor, vals: torch.Tensor,
                  mode="f64_plain", stream=None):
    """(sign, log|det A|) of a CSR matrix as 0-d FP64 CUDA tensors: the diagonal
    blocks of its block triangular form condensed on the GPU (ld_logdet_sparse).
    The arrays may live on the host or on the GPU; the call waits for the stream."""
    row_ptr, col_idx = _csr_arrays(row_ptr, col_idx)
    vals = vals.contiguous()
    n = row_ptr.numel() - 1
    if n < 0:
        raise ValueError("row_ptr needs n + 1 entries")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    code = _lib.ld_logdet_sparse(row_ptr.data_ptr(), col_idx.data_ptr(), vals.data_ptr(),
                                 _dtype_code(vals), n, _mode_code(mode), _stream_handle(stream),
                                 out.data_ptr(), out.data_ptr() + 8)
    _lib.check("ld_logdet_sparse", code)
    return out[0], out[1]


def sparse_blocks(row_ptr: torch.Tensor, col_idx: torch.Tensor):
    """The structure analysis of logdet_sparse on the host: (col_of_row,
    block_of_row, nblocks) as CPU tensors and an int; nblocks = -1 when the matrix
    has no complete transversal (structurally singular)."""
    import ctypes
    row_ptr, col_idx = _csr_arrays(row_ptr.cpu(), col_idx.cpu())
    n = row_ptr.numel() - 1
    cor = torch.empty(max(n, 0), dtype=torch.int64)
    blk = torch.empty(max(n, 0), dtype=torch.int64)
    nb = ctypes.c_int64()
    code = _lib.ld_sparse_blocks(row_ptr.data_ptr(), col_idx.data_ptr(), n, cor.data_ptr(),
                                 blk.data_ptr(), ctypes.addressof(nb))
    _lib.check("ld_sparse_blocks", code)
    return cor, blk, nb.value

