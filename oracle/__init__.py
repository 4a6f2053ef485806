"""Oracle: plain CPU FP64 reference for the condensation log-determinant.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA path in
``paper_1811_08057_gb300`` never imports it, and it never imports that package.

Contents
--------
``logdet``            sign and log|det A| by the condensation sweep (Eqs. (2)-(3),
                      Sec. 2.2, Fig. 6 with one process), written in plain C
                      (``condense_oracle.c``), FP64, one FMA per minor.
``condense_once``     one step of Eq. (2) around an arbitrary pivot (k, l).
``logdet_batched``    ``logdet`` over a list of matrices.
``grad_logabs``       d log|det A| / dA = A^{-T}, the plain definition
                      (Jacobi's formula), via a library inverse in FP64.
``exact``             exact-integer and exact-rational references for small n
                      (Leibniz expansion, rational condensation).
"""
from .core import (  # noqa: F401
    build,
    condense_once,
    grad_logabs,
    library_path,
    logdet,
    logdet_batched,
)
from . import exact  # noqa: F401
