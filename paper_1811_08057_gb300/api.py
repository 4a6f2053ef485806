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
    """(sign, log|det A|) as 0-d FP64 CUDA tensors (no host synchronisation)."""
    _check_matrix(A)
    n = A.shape[0]
    lda = max(A.stride(0), 1) if n > 0 else 1
    out = torch.empty(2, dtype=torch.float64, device=A.device)
    code = _lib.ld_logdet(A.data_ptr(), _dtype_code(A), n, lda, _mode_code(mode),
                          _stream_handle(stream), out.data_ptr(), out.data_ptr() + 8)
    _lib.check("ld_logdet", code)
    return out[0], out[1]


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
    f64 = mode in (_lib.LD_F64_PLAIN, _lib.LD_F64_BLOCKED)
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
    BatchedInputs) in one persistent launch. Returns (signs, logabs) FP64 tensors."""
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
