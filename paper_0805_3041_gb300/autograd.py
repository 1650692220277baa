"""Differentiable solves of -div(k grad u) = f through the multigrid F-cycle.

Forward: u = A(k)^{-1} f by F-cycles (mg_solve).  Backward, for an upstream
gradient g = dL/du: the adjoint solve A(k)^T lambda = g runs the transposed
F-cycle (mg_solve_adjoint: the cycle's steps in reverse order, each transposed);
then dL/df = lambda and dL/dk_c = -sum over the edges e of cell c of
(dw_e/dk_c)(u_p - u_q)(lambda_p - lambda_q) (mg_grad_coeff), the derivative of
lambda^T A(k) u for edge weights linear in k.  Every step runs in the library's
CUDA kernels; this module only wires them into torch.autograd.
"""
from __future__ import annotations

import torch

from . import inputs
from .binding import Solver


def _spec(k, n, h, dim):
    return inputs.ProblemSpec(name="diffusion", dim=dim, n=n, periodic_y=False, kind=inputs.CELL, h=h, k=k)


class MGDiffusionSolve(torch.autograd.Function):
    """u = solve(k, f): k per cell, f per node (Dirichlet entries ignored), both float64 CUDA tensors."""

    @staticmethod
    def forward(ctx, k, f, levels, smoother, omega, precision, tol, max_cycles):
        dim = f.dim()
        n = tuple(reversed(f.shape)) + (1,) * (3 - f.dim())
        h = tuple(1.0 / (m - 1) if m > 1 else 1.0 for m in n)
        s = Solver(_spec(k.detach().contiguous(), n, h, dim), levels=levels, smoother=smoother, omega=omega,
                   precision=precision, max_cycles=max_cycles, device=f.device)
        u, info = s.solve(f.detach(), tol=tol)
        if info["status"] != "MG_OK":
            raise RuntimeError(f"forward multigrid solve did not converge: {info['status']}, relres {info['relres']:.2e}")
        ctx.solver = s
        ctx.tol = tol
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        s = ctx.solver
        lam, info = s.solve_adjoint(grad_u.detach().contiguous(), tol=ctx.tol)
        if info["status"] != "MG_OK":
            raise RuntimeError(f"adjoint multigrid solve did not converge: {info['status']}")
        grad_k = s.grad_coeff(u, lam) if ctx.needs_input_grad[0] else None
        grad_f = lam if ctx.needs_input_grad[1] else None
        return grad_k, grad_f, None, None, None, None, None, None


def diffusion_solve(k, f, levels, smoother="rbgs", omega=1.0, precision="fp64", tol=1e-12, max_cycles=100):
    """Differentiable multigrid solve of -div(k grad u) = f on the unit square / cube with zero
    Dirichlet data; k has one value per cell, f one per node."""
    return MGDiffusionSolve.apply(k, f, levels, smoother, omega, precision, tol, max_cycles)
