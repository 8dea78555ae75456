"""Differentiable sum of the k smallest eigenvalues with respect to the potential.

E(V) = sum_{i<k} lambda_i(A(V)), A(V) = -Laplacian_h + diag(V). By the Hellmann-Feynman theorem
dE/dV_p = sum_{i<k} x_i(p)^2 for unit-norm eigenvectors, provided lambda_k < lambda_{k+1}. The forward pass is
ppcg_solve; the backward pass is the library's density kernel (ppcg_energy_gradient) on the returned vectors.
"""
from __future__ import annotations

import ctypes

import torch

from . import ppcg_energy_gradient


class _SmallestEigsum(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, solver, X0, tol):
        solver.set_potential(V.detach())
        lam, X, res, st = solver.solve(X0, tol)
        if st["converged"] != 1:
            raise RuntimeError(f"PPCG did not converge (max residual {st['max_res']:.3e})")
        ctx.solver = solver
        ctx.save_for_backward(X)
        out = torch.tensor(float(lam.sum()), dtype=torch.float64, device=V.device)
        ctx.lam = lam
        return out

    @staticmethod
    def backward(ctx, g):
        (X,) = ctx.saved_tensors
        solver = ctx.solver
        grad = torch.empty(solver.n, dtype=torch.float64, device=X.device)
        ppcg_energy_gradient(solver.handle, X.data_ptr(), solver.n, solver.k, float(g.item()), grad.data_ptr())
        return grad, None, None, None


def smallest_eigsum(V: torch.Tensor, solver, X0, tol: float = 1e-10) -> torch.Tensor:
    """E = sum of the k smallest eigenvalues of -Laplacian + diag(V); differentiable in V (Hellmann-Feynman)."""
    return _SmallestEigsum.apply(V, solver, X0, tol)
