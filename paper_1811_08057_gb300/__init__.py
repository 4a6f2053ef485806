"""GB300 (sm_103a) matrix-condensation log-determinant.

Salem-Said condensation with max-abs pivoting in the pivot row (Dong, Barnett,
Dhall, "Parallel Matrix Condensation for Calculating Log-Determinant of Large
Matrix", Eqs. (2)-(3), Sec. 2.2-2.4). All arithmetic runs in liblogdet's CUDA
kernels; this package marshals torch tensors into the C ABI.

    sign, logabs = logdet(A, mode="f64_plain")
"""
from __future__ import annotations

from ._lib import (  # noqa: F401
    LD_DTYPE_F32,
    LD_DTYPE_F64,
    MODES,
    LogdetError,
    check,
    ld_factors_size,
    ld_logdet,
    ld_logdet_backward,
    ld_logdet_batched,
    ld_logdet_factor,
    ld_logdet_variant,
    ld_status_string,
    ld_version,
    load,
)
from .api import (  # noqa: F401
    BatchedInputs,
    Factors,
    LogAbsDet,
    logabsdet,
    logdet_backward,
    logdet,
    logdet_batched,
    logdet_factor,
    logdet_sparse,
    logdet_variant,
    logdet_variant_factor,
    parse_factors,
    sparse_blocks,
)
