"""GB300-native solve phase of the two-grid algebraic multiscale (AMS)
preconditioner (arXiv 2606.04864): PCG on sparse SPD systems with local
subdomain solves plus a spectral coarse correction, all in hand-written
CUDA for sm_103a behind the C ABI in ``include/ams.h``."""

from ._lib import AmsError, lib  # noqa: F401
from .solver import AmsBatchedSolver, AmsSolver, partition  # noqa: F401

__all__ = ["AmsSolver", "AmsBatchedSolver", "AmsError", "lib", "partition"]
