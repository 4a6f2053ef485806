"""ctypes front end of the C oracle (test infrastructure only).

The C file is compiled with gcc on first use (or by ``build()``), with
``-ffp-contract=off`` so that the only fused multiply-add is the explicit one in
each Eq. (2) minor.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "condense_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_condense.so")
_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB


def compile_c(src: str, out: str) -> str:
    """gcc the oracle source ``src`` into the shared library ``out``."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-D_POSIX_C_SOURCE=200809L", "-pthread", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def source_path() -> str:
    return _SRC


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build``. Returns the library path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_c(_SRC, _LIB)
    return _LIB


def _bind(path: str):
    lib = ctypes.CDLL(path)
    i64, dbl = ctypes.c_int64, ctypes.c_double
    pd = ctypes.POINTER(dbl)
    pi = ctypes.POINTER(i64)
    lib.oracle_logdet.argtypes = [pd, i64, i64, i64, ctypes.c_int, pd, pd, pi, pd, pi]
    lib.oracle_logdet.restype = ctypes.c_int
    lib.oracle_logdet_ex.argtypes = [pd, i64, i64, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     pd, pd, pi, pd, pi]
    lib.oracle_logdet_ex.restype = ctypes.c_int
    lib.oracle_condense_once.argtypes = [pd, i64, i64, i64, i64, pd, pd]
    lib.oracle_condense_once.restype = ctypes.c_int
    return lib


def _load(path: str | None = None):
    """The default oracle library, or (for mutation tests) one built elsewhere."""
    global _lib
    if path is not None:
        return _bind(path)
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


@dataclass
class OracleResult:
    sign: float
    logabs: float
    piv_label: np.ndarray  # int64[n], original column label of each pivot
    piv_value: np.ndarray  # float64[n], signed pivot of each step
    steps: int


def _as_f64(A) -> np.ndarray:
    A = np.asarray(A, dtype=np.float64)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square")
    return np.ascontiguousarray(A)


# pivot-column rules (oracle_logdet_ex): the paper's max |a_kj| (Sec. 2.2) and the
# two rules of earlier work it names (Sec. 1)
RULES = {"max_abs": 0, "closest_to_one": 1, "first_nonzero": 2}


def logdet(A, *, max_steps: int = -1, nthreads: int = 1, rule: str = "max_abs",
           factor: str = "row", _library: str | None = None) -> OracleResult:
    """sign(det A), log|det A| and the pivot sequence, FP64 (Eqs. (2)-(3), Sec. 2.2).

    rule: pivot column "max_abs" (the paper's), "closest_to_one" or
    "first_nonzero" (Sec. 1); factor: the pivot factored out of the "row" (the
    paper's) or the "column" (Sec. 2.3).
    """
    lib = _load(_library)
    A = _as_f64(A)
    n = A.shape[0]
    sign = ctypes.c_double()
    logabs = ctypes.c_double()
    steps = ctypes.c_int64()
    lab = np.empty(max(n, 1), dtype=np.int64)
    val = np.empty(max(n, 1), dtype=np.float64)
    pd = ctypes.POINTER(ctypes.c_double)
    pi = ctypes.POINTER(ctypes.c_int64)
    if factor not in ("row", "column"):
        raise ValueError("factor must be 'row' or 'column'")
    if rule == "max_abs" and factor == "row":
        rc = lib.oracle_logdet(A.ctypes.data_as(pd), n, n, max_steps, int(nthreads),
                               ctypes.byref(sign), ctypes.byref(logabs),
                               lab.ctypes.data_as(pi), val.ctypes.data_as(pd), ctypes.byref(steps))
    else:
        rc = lib.oracle_logdet_ex(A.ctypes.data_as(pd), n, n, max_steps, int(nthreads),
                                  RULES[rule], 1 if factor == "column" else 0,
                                  ctypes.byref(sign), ctypes.byref(logabs),
                                  lab.ctypes.data_as(pi), val.ctypes.data_as(pd),
                                  ctypes.byref(steps))
    if rc != 0:
        raise RuntimeError(f"oracle_logdet failed with code {rc}")
    return OracleResult(sign.value, logabs.value, lab[:n].copy(), val[:n].copy(), steps.value)


def condense_once(A, k: int, l: int, _library: str | None = None):
    """One Eq. (2) step around pivot (k, l), 0-based, row k factored (Eq. (3)).

    Returns (B, factor) with det A = factor * det B.
    """
    lib = _load(_library)
    A = _as_f64(A)
    m = A.shape[0]
    B = np.empty((m - 1, m - 1), dtype=np.float64)
    factor = ctypes.c_double()
    pd = ctypes.POINTER(ctypes.c_double)
    rc = lib.oracle_condense_once(A.ctypes.data_as(pd), m, m, int(k), int(l),
                                  B.ctypes.data_as(pd), ctypes.byref(factor))
    if rc != 0:
        raise ValueError(f"oracle_condense_once failed with code {rc}")
    return B, factor.value


def logdet_batched(mats, *, nthreads: int = 1):
    """``logdet`` of each matrix of a list (the batched path computes exactly this)."""
    return [logdet(A, nthreads=nthreads) for A in mats]


def grad_logabs(A, g: float = 1.0) -> np.ndarray:
    """g * d log|det A| / dA = g * A^{-T} (Jacobi's formula), FP64 library inverse."""
    A = _as_f64(A)
    return float(g) * np.linalg.inv(A).T
