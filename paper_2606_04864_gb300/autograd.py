"""Differentiable AMS solve: torch.autograd.Function around the C ABI.

Forward: u = A^{-1} f by AMS-preconditioned CG (ams_solve).
Backward (hand-written): the adjoint solve lambda = A^{-1} (dL/du) with the
same preconditioner (A is symmetric), then the sampled outer product on A's
pattern, dL/dA_vals[e] = -sum_k lambda_k[row_e] u_k[col_e], and dL/df =
lambda (ams_solve_adjoint).  Both run in the CUDA library.
"""

from __future__ import annotations

import torch

from .solver import AmsSolver


class AmsSolveFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, f, solver: AmsSolver, rtol: float, adjoint_rtol: float):
        if not solver.device:
            raise ValueError("AmsSolveFunction needs a solver built with device=True")
        if vals.shape != (solver.nnz,):
            raise ValueError(f"vals must hold the {solver.nnz} CSR values of the solver's pattern")
        # the solve uses these values (device to device); the preconditioner
        # built at setup is kept, so CG stays exact for the new matrix and
        # converges fastest while it stays close to the setup matrix
        solver.set_matrix_values(vals.detach())
        u, its, rel = solver.solve(f, rtol)
        ctx.solver = solver
        ctx.adjoint_rtol = adjoint_rtol
        ctx.f_shape = f.shape
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        solver: AmsSolver = ctx.solver
        lam, dvals, its = solver.solve_adjoint(grad_u.contiguous(), u, ctx.adjoint_rtol,
                                               want_dvals=ctx.needs_input_grad[0])
        grad_f = lam.reshape(ctx.f_shape) if ctx.needs_input_grad[1] else None
        return dvals, grad_f, None, None, None


def ams_solve(vals: torch.Tensor, f: torch.Tensor, solver: AmsSolver, rtol: float = 1e-8,
              adjoint_rtol: float | None = None) -> torch.Tensor:
    """u = A(vals)^{-1} f, differentiable in ``vals`` and ``f``.

    ``solver`` must have been set up (device=True) on a matrix with the
    CSR pattern of ``vals``.  Each call first loads ``vals`` into the
    solver (``set_matrix_values``), so the forward solves with the matrix
    these values define and the backward's adjoint solve and dL/dA use the
    same matrix; the preconditioner stays the one built at setup."""
    return AmsSolveFunction.apply(vals, f, solver, rtol, rtol if adjoint_rtol is None else adjoint_rtol)
