"""Differentiable solve u = A(alpha)^{-1} f as a torch.autograd.Function.

Forward: one library solve (PCG + V-cycle, FP64 or mixed with FP64
refinement).  Backward: the adjoint solve A lambda = dL/du with the same
handle and V-cycle (A is symmetric: a(w, v) = a(v, w), and so is the V-cycle
preconditioner, Remark 6 of arXiv 2205.05840), then dL/df = lambda and
dL/dalpha = -lambda^T K u with K the alpha-free curl-curl matrix
(library entry point ndmg_grad_alpha).  With a coefficient per hexahedron
(solve_field) the same adjoint gives dL/dalpha_T = -lambda^T K_T u for every
cell (ndmg_grad_alpha_field).  Marshalling only: every step runs in the CUDA
library.
"""
from __future__ import annotations

import torch

from . import ndmg


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f: torch.Tensor, alpha: torch.Tensor, solver: "ndmg.Solver", tol: float, maxit: int):
        a = float(alpha.detach())
        if solver.alpha is None or abs(a - solver.alpha) > 0.0:
            solver.set_alpha(a)
        u = torch.zeros_like(f)
        solver.solve(f.detach().contiguous(), u, tol=tol, maxit=maxit)
        ctx.solver, ctx.tol, ctx.maxit, ctx.alpha = solver, tol, maxit, a
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, gu: torch.Tensor):
        (u,) = ctx.saved_tensors
        S = ctx.solver
        if S.alpha is None or abs(ctx.alpha - S.alpha) > 0.0:
            S.set_alpha(ctx.alpha)
        lam = torch.zeros_like(u)
        S.solve(gu.detach().contiguous().to(u.dtype), lam, tol=ctx.tol, maxit=ctx.maxit)
        dalpha = S.grad_alpha(lam, u)
        if isinstance(dalpha, list):
            # a batch of right-hand sides shares the one alpha: its gradient is
            # the sum of the per-right-hand-side -lambda_r^T K u_r
            dalpha = sum(dalpha)
        return lam, torch.tensor(dalpha, dtype=torch.float64), None, None, None


def solve(f: torch.Tensor, alpha: torch.Tensor, solver: "ndmg.Solver", tol: float = 1e-10, maxit: int = 500):
    """u(f, alpha) with gradients to f and alpha (alpha: 0-d float64 tensor)."""
    return _Solve.apply(f, alpha, solver, tol, maxit)


class _SolveField(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f: torch.Tensor, alpha_cells: torch.Tensor, solver: "ndmg.Solver", tol: float, maxit: int):
        a = alpha_cells.detach().to("cpu", torch.float64).contiguous()
        solver.set_alpha_field(a)
        u = torch.zeros_like(f)
        solver.solve(f.detach().contiguous(), u, tol=tol, maxit=maxit)
        ctx.solver, ctx.tol, ctx.maxit, ctx.field = solver, tol, maxit, a
        ctx.adev = alpha_cells.device
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, gu: torch.Tensor):
        (u,) = ctx.saved_tensors
        S = ctx.solver
        S.set_alpha_field(ctx.field)      # the handle may have moved on since the forward pass
        lam = torch.zeros_like(u)
        S.solve(gu.detach().contiguous().to(u.dtype), lam, tol=ctx.tol, maxit=ctx.maxit)
        dfield = S.grad_alpha_field(lam, u)
        return lam, dfield.to(ctx.adev), None, None, None


def solve_field(f: torch.Tensor, alpha_cells: torch.Tensor, solver: "ndmg.Solver", tol: float = 1e-10,
                maxit: int = 500):
    """u(f, alpha) for a coefficient per finest-level hexahedron (alpha_cells:
    n^3 float64 values, cell (i, j, k) at (k n + j) n + i), with gradients to f
    and to every cell coefficient."""
    return _SolveField.apply(f, alpha_cells, solver, tol, maxit)
