"""ctypes binding of liblogdet: the C entry points under the same names.

Argument marshalling only. The library must have been built (``build.build()``);
loading fails loudly otherwise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

# ld_mode
LD_F64_PLAIN = 0
LD_F64_BLOCKED = 1
LD_F32_PLAIN = 2
LD_F32_TF32 = 3
LD_F32_3XTF32 = 4
LD_F32_BF16X3 = 5
LD_F64_OZAKI = 6
MODES = {
    "f64_plain": LD_F64_PLAIN,
    "f64_blocked": LD_F64_BLOCKED,
    "f32_plain": LD_F32_PLAIN,
    "f32_tf32": LD_F32_TF32,
    "f32_3xtf32": LD_F32_3XTF32,
    "f32_bf16x3": LD_F32_BF16X3,
    "f64_ozaki": LD_F64_OZAKI,
}
F64_MODES = (LD_F64_PLAIN, LD_F64_BLOCKED, LD_F64_OZAKI)
# ld_pivot_rule, ld_factor_side
PIVOT_RULES = {"max_abs": 0, "closest_to_one": 1, "first_nonzero": 2}
FACTOR_SIDES = {"row": 0, "column": 1}
# ld_dtype
LD_DTYPE_F64 = 0
LD_DTYPE_F32 = 1
# ld_status
STATUS = {0: "LD_OK", 1: "LD_ERR_INVALID_ARG", 2: "LD_ERR_UNSUPPORTED", 3: "LD_ERR_ALLOC",
          4: "LD_ERR_CUDA", 5: "LD_ERR_TIMEOUT"}
LD_OK = 0
LD_ERR_INVALID_ARG = 1

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_sz = ctypes.c_size_t
_pd = ctypes.c_void_p  # double* (host or device address as an integer)

SIGNATURES = {
    "ld_logdet": ([_vp, _int, _i64, _i64, _int, _vp, _pd, _pd], _int),
    "ld_factors_size": ([_i64, _int], _sz),
    "ld_logdet_variant": ([_vp, _int, _i64, _i64, _int, _int, _int, _vp, _vp, _pd, _pd], _int),
    "ld_logdet_factor": ([_vp, _int, _i64, _i64, _int, _vp, _vp, _pd, _pd], _int),
    "ld_logdet_backward": ([_vp, _vp, _vp, _i64, _vp], _int),
    "ld_logdet_batched": ([_vp, _int, _vp, _vp, _i64, _i64, _int, _vp, _vp, _vp], _int),
    "ld_logdet_batched_factor": ([_vp, _int, _vp, _vp, _i64, _i64, _int, _vp, _vp, _vp, _vp],
                                 _int),
    "ld_logdet_backward_batched": ([_vp, _i64, _i64, _int, _vp, _vp, _i64, _vp], _int),
    "ld_rankb_update": ([_int, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp], _int),
    "ld_logdet_noalloc": ([_vp, _int, _i64, _i64, _vp, _pd, _pd], _int),
    "ld_logdet_sparse": ([_vp, _vp, _vp, _int, _i64, _int, _vp, _pd, _pd], _int),
    "ld_sparse_blocks": ([_vp, _vp, _i64, _vp, _vp, _vp], _int),
    "ld_rowblock_factor": ([_vp, _int, _vp, _i64, _vp, _vp], _int),
    "ld_rowblock_update": ([_vp, _int, _i64, _i64, _i64, _vp, _vp, _vp, _vp], _int),
    "ld_profile_start": ([ctypes.c_char_p], _int),
    "ld_profile_stop": ([], _int),
    "ld_profile_query": ([ctypes.c_char_p, _vp, _vp], _int),
    "ld_profile_work": ([ctypes.c_char_p, _vp, _vp], _int),
    "ld_profile_classes": ([_vp, _i64], _int),
    "ld_set_tuning": ([ctypes.c_char_p, _i64], _int),
    "ld_tune": ([_vp, _i64, _int, _vp], _int),
    "ld_tune_save": ([ctypes.c_char_p], _int),
    "ld_tune_load": ([ctypes.c_char_p], _int),
    "ld_get_tuning": ([ctypes.c_char_p, _vp], _int),
    "ld_status_string": ([_int], ctypes.c_char_p),
    "ld_version": ([], ctypes.c_char_p),
}


class LogdetError(RuntimeError):
    def __init__(self, func: str, code: int):
        self.code = code
        super().__init__(f"{func} returned {STATUS.get(code, code)}")


def library_path() -> str:
    return _build.LIB_PATH


def load(path: str | None = None):
    """Load liblogdet.so (building it first if its sources are newer)."""
    global _lib
    with _lock:
        if _lib is None or path is not None:
            p = path or _build.build()
            if not os.path.exists(p):
                raise RuntimeError(f"liblogdet is not built ({p} missing)")
            lib = ctypes.CDLL(p)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            if path is not None:
                return lib
            _lib = lib
    return _lib


def header_symbols(header: str | None = None):
    """Names of the functions that include/logdet.h declares."""
    header = header or os.path.join(_build.INCLUDE, "logdet.h")
    with open(header) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ld_[a-z_0-9]+)\s*\(", text)))


def check(func: str, code: int):
    if code != 0:
        raise LogdetError(func, code)


# Same-name thin wrappers (integers are device/host addresses).
def ld_logdet(A, a_dtype, n, lda, mode, stream, sign, logabs) -> int:
    return load().ld_logdet(A, a_dtype, n, lda, mode, stream, sign, logabs)


def ld_logdet_variant(A, a_dtype, n, lda, mode, rule, side, stream, factors, sign, logabs) -> int:
    return load().ld_logdet_variant(A, a_dtype, n, lda, mode, rule, side, stream, factors, sign,
                                    logabs)


def ld_rowblock_factor(row, dtype, labels, m, step, stream) -> int:
    return load().ld_rowblock_factor(row, dtype, labels, m, step, stream)


def ld_rowblock_update(F, dtype, rows, ldf, m, r, labels, step, stream) -> int:
    return load().ld_rowblock_update(F, dtype, rows, ldf, m, r, labels, step, stream)


def ld_factors_size(n, mode) -> int:
    return load().ld_factors_size(n, mode)


def ld_logdet_factor(A, a_dtype, n, lda, mode, stream, factors, sign, logabs) -> int:
    return load().ld_logdet_factor(A, a_dtype, n, lda, mode, stream, factors, sign, logabs)


def ld_logdet_backward(factors, g, grad, ldg, stream) -> int:
    return load().ld_logdet_backward(factors, g, grad, ldg, stream)


def ld_logdet_batched(A_ptrs, a_dtype, n, lda, count, n_max, mode, stream, signs, logabs) -> int:
    return load().ld_logdet_batched(A_ptrs, a_dtype, n, lda, count, n_max, mode, stream, signs,
                                    logabs)


def ld_logdet_batched_factor(A_ptrs, a_dtype, n, lda, count, n_max, mode, stream, factors, signs,
                             logabs) -> int:
    return load().ld_logdet_batched_factor(A_ptrs, a_dtype, n, lda, count, n_max, mode, stream,
                                           factors, signs, logabs)


def ld_logdet_backward_batched(factors, count, n, mode, g, grads, ldg, stream) -> int:
    return load().ld_logdet_backward_batched(factors, count, n, mode, g, grads, ldg, stream)


def ld_rankb_update(mode, M, N, K, A, lda, B, ldb, D, ldd, stream) -> int:
    return load().ld_rankb_update(mode, M, N, K, A, lda, B, ldb, D, ldd, stream)


def ld_logdet_noalloc(A, a_dtype, n, lda, stream, sign, logabs) -> int:
    return load().ld_logdet_noalloc(A, a_dtype, n, lda, stream, sign, logabs)


def ld_logdet_sparse(row_ptr, col_idx, vals, v_dtype, n, mode, stream, sign, logabs) -> int:
    return load().ld_logdet_sparse(row_ptr, col_idx, vals, v_dtype, n, mode, stream, sign, logabs)


def ld_sparse_blocks(row_ptr, col_idx, n, col_of_row, block_of_row, nblocks) -> int:
    return load().ld_sparse_blocks(row_ptr, col_idx, n, col_of_row, block_of_row, nblocks)


def ld_profile_start(kernel=None) -> int:
    return load().ld_profile_start(kernel.encode() if kernel else None)


def ld_profile_stop() -> int:
    return load().ld_profile_stop()


def ld_profile_query(kernel=None):
    """(launches, total_ms) of a kernel class since ld_profile_start."""
    n = ctypes.c_int64()
    t = ctypes.c_double()
    code = load().ld_profile_query(kernel.encode() if kernel else None, ctypes.addressof(n),
                                   ctypes.addressof(t))
    check("ld_profile_query", code)
    return n.value, t.value


def ld_profile_work(kernel=None):
    """(bytes, flops) declared by the launches of a kernel class since ld_profile_start."""
    b = ctypes.c_double()
    f = ctypes.c_double()
    code = load().ld_profile_work(kernel.encode() if kernel else None, ctypes.addressof(b),
                                  ctypes.addressof(f))
    check("ld_profile_work", code)
    return b.value, f.value


def ld_profile_classes():
    buf = ctypes.create_string_buffer(4096)
    check("ld_profile_classes", load().ld_profile_classes(ctypes.addressof(buf), 4096))
    v = buf.value.decode()
    return [x for x in v.split(",") if x]


def ld_set_tuning(name: str, value: int) -> int:
    return load().ld_set_tuning(name.encode(), int(value))


def ld_get_tuning(name: str) -> int:
    v = ctypes.c_int64()
    check("ld_get_tuning", load().ld_get_tuning(name.encode(), ctypes.addressof(v)))
    return v.value


def ld_tune(sizes, mode, stream=None) -> int:
    """Autotunes the table for these matrix sizes (a list of ints) in `mode`."""
    arr = (ctypes.c_int64 * len(sizes))(*[int(x) for x in sizes])
    return load().ld_tune(ctypes.addressof(arr), len(sizes), mode, stream)


def ld_tune_save(path=None) -> int:
    return load().ld_tune_save(path.encode() if path else None)


def ld_tune_load(path=None) -> int:
    return load().ld_tune_load(path.encode() if path else None)


def ld_status_string(code) -> str:
    return load().ld_status_string(code).decode()


def ld_version() -> str:
    return load().ld_version().decode()
