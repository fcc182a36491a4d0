"""Seeded synthetic Darcy workloads (input generation only).

This package builds the inputs that both the CPU oracle and the GPU library
consume: two-point flux (TPFA) Darcy matrices in CSR form, Gaussian-random-
field and channelised permeabilities, regular block partitions, right-hand
sides and observation sets.  It holds none of the preconditioner's
arithmetic (no restriction, eigenproblem, coarse operator or Krylov step), so
the oracle and the CUDA path can share it without sharing method code.

The paper's own test matrices come from an RT0 mixed discretisation of a
pure-Neumann heat problem with channel and fracture permeability images
(Section 5); those images and matrices are not available, so these
generators stand in for them with the same structure: a sparse SPD M-matrix
from an elliptic operator on a Cartesian grid, heterogeneous coefficients
with high contrast, and a regular graph partition.
"""

from .darcy import (  # noqa: F401
    Workload,
    block_partition,
    channel_field,
    grf_logk,
    tpfa_csr,
    tpfa_face_list,
    tpfa_values_from_logk,
    make_grf2d_64,
    make_channels2d_1024,
    make_grf3d_128_rhs32,
    make_batch48_uneven,
    make_grf3d_96_adjoint,
    make_small_2d,
    make_small_3d,
    make_from_logk,
)
