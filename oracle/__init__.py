"""CPU oracle for the two-grid algebraic multiscale (AMS) preconditioned CG.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64
restatement of the paper's method used to check the CUDA library.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
and reference legs) may import it; the library in
``paper_2606_04864_gb300`` never does, and it shares no code with it.
"""

from .ams_oracle import (  # noqa: F401
    OracleAMS,
    index_maps,
    local_matrices,
    local_eigenpairs,
    coarse_basis,
    coarse_matrix,
    pcg,
    adjoint_gradient,
    csr_to_scipy,
)
