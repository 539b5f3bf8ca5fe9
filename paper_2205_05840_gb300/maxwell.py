"""Implicit time stepping of Maxwell's equations on the multigrid solver
(Sec. 1, eq. (Maxwell timestep)).

Eliminating H from the first-order system gives eps E_tt + sigma E_t +
curl(mu^{-1} curl E) = J_t.  The three-level implicit scheme

    eps M (E+ - 2E + E-)/dt^2 + sigma M (E+ - E-)/(2 dt) + K (E+ + 2E + E-)/(4 mu) = F

leaves at every time level the model problem a(E+, v) = (rhs, v) with
alpha = dt^2/(4 mu) and beta = eps + sigma dt/2, which is the operator of
eq. (Maxwell timestep):

    rhs = (2 eps M - dt^2/(2 mu) K) E + ((sigma dt/2 - eps) M - dt^2/(4 mu) K) E- + dt^2 F.

One step is two library pencil applications (ndmg_pencil) for the
right-hand side, one vector update for the warm start E+ ~ 2E - E-
(ndmg_axpby), and one preconditioned solve (ndmg_solve); a batch of nrhs
independent fields (different sources) steps together through the batched
path.  With sigma = 0 and F = 0 the scheme conserves
eps/dt^2 |E+ - E|_M^2 + 1/(4 mu) |E+ + E|_K^2.
"""
from __future__ import annotations

import torch

from . import ndmg


def step_coefficients(dt: float, eps: float, sigma: float, mu: float) -> tuple[float, float]:
    """(alpha, beta) of the per-step operator, eq. (Maxwell timestep)."""
    return dt * dt / (4.0 * mu), eps + 0.5 * sigma * dt


class ImplicitMaxwell:
    """Time stepper for nrhs fields on an n^3 grid of the cube of side L."""

    def __init__(self, n: int, dt: float, eps: float = 1.0, sigma: float = 0.0, mu: float = 1.0, L: float = 1.0,
                 n_coarsest: int = 4, m: int = 2, precision: int = ndmg.PREC_MIXED_FP16, nrhs: int = 1,
                 tol: float = 1e-8, maxit: int = 200):
        self.dt, self.eps, self.sigma, self.mu, self.tol, self.maxit = dt, eps, sigma, mu, tol, maxit
        alpha, beta = step_coefficients(dt, eps, sigma, mu)
        self.solver = ndmg.Solver(n, n_coarsest=n_coarsest, L=L, alpha=alpha, beta=beta, m=m,
                                  precision=precision, nrhs=nrhs)
        self.size = self.solver.num_dofs() * nrhs
        self._rhs = torch.empty(self.size, dtype=torch.float64, device="cuda")
        self.iterations: list[int] = []

    def rhs(self, E: torch.Tensor, E_prev: torch.Tensor, load: torch.Tensor | None = None) -> torch.Tensor:
        """Right-hand side of the step from E (level n) and E_prev (level n-1);
        `load` is the load vector F of the source term (or None)."""
        S, dt, eps, sig, mu = self.solver, self.dt, self.eps, self.sigma, self.mu
        r = self._rhs
        if load is None:
            S.pencil(-dt * dt / (2.0 * mu), 2.0 * eps, E, r)
        else:
            S.axpby(dt * dt, load, 0.0, r)
            S.pencil(-dt * dt / (2.0 * mu), 2.0 * eps, E, r, g=r)
        S.pencil(-dt * dt / (4.0 * mu), 0.5 * sig * dt - eps, E_prev, r, g=r)
        return r

    def step(self, E: torch.Tensor, E_prev: torch.Tensor, load: torch.Tensor | None = None,
             out: torch.Tensor | None = None) -> torch.Tensor:
        """E at the next time level, written to `out` (which may be E_prev, not E)."""
        if out is E:
            raise ValueError("out must not be E (it is read for the warm start)")
        S = self.solver
        r = self.rhs(E, E_prev, load)
        if out is None:
            out = torch.empty_like(E)
        if out is not E_prev:
            S.axpby(1.0, E_prev, 0.0, out)
        S.axpby(2.0, E, -1.0, out)              # warm start 2E - E_prev
        _, it, _ = S.solve(r, out, tol=self.tol, maxit=self.maxit)
        self.iterations.append(it)
        return out

    def run(self, E_prev: torch.Tensor, E: torch.Tensor, loads) -> list[torch.Tensor]:
        """Levels 2 .. 1 + len(loads) from E^0 = E_prev and E^1 = E (both kept)."""
        out = []
        for F in loads:
            E_new = self.step(E, E_prev, F)
            out.append(E_new)
            E_prev, E = E, E_new
        return out
