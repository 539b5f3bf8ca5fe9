"""FP64 CPU oracle: implicit time stepping of Maxwell's equations.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library.

What it follows (arXiv 2205.05840, Sec. 1, eq. (Maxwell timestep)): eliminating
H from the first-order Maxwell system gives the second-order equation

    eps E_tt + sigma E_t + curl(mu^{-1} curl E) = J_t,

and an implicit step leaves, at every time level, the model problem with
alpha = dt^2 / (4 mu) and beta = eps + sigma dt / 2.  The paper does not state
the right-hand side; the reading here is the three-level scheme that produces
exactly that operator (average-acceleration Newmark): with K the alpha-free
curl-curl matrix and M the mass matrix,

    eps M (E+ - 2E + E-) / dt^2 + sigma M (E+ - E-) / (2 dt)
        + K (E+ + 2E + E-) / (4 mu) = F,

i.e.  (dt^2/(4 mu) K + (eps + sigma dt/2) M) E+ =
          (2 eps M - dt^2/(2 mu) K) E + ((sigma dt/2 - eps) M - dt^2/(4 mu) K) E-
          + dt^2 F.

Each step is solved directly (sparse LU): the oracle of the time stepper does
not depend on the multigrid oracle.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import hcurl


def step_coefficients(dt: float, eps: float, sigma: float, mu: float) -> tuple[float, float]:
    """(alpha, beta) of the per-step operator, eq. (Maxwell timestep)."""
    return dt * dt / (4.0 * mu), eps + 0.5 * sigma * dt


class ImplicitMaxwell:
    """The three-level implicit scheme on an n^3 grid of [0, L]^3."""

    def __init__(self, n: int, L: float, dt: float, eps: float = 1.0, sigma: float = 0.0, mu: float = 1.0):
        self.n, self.L, self.dt, self.eps, self.sigma, self.mu = n, L, dt, eps, sigma, mu
        self.K, self.M = hcurl.assemble_parts(n, L)
        self.alpha, self.beta = step_coefficients(dt, eps, sigma, mu)
        self.A = (self.alpha * self.K + self.beta * self.M).tocsc()
        self._lu = spla.splu(self.A)

    def rhs(self, E: np.ndarray, E_prev: np.ndarray, F: np.ndarray | None = None) -> np.ndarray:
        dt, eps, sig, mu = self.dt, self.eps, self.sigma, self.mu
        r = 2.0 * eps * (self.M @ E) - dt * dt / (2.0 * mu) * (self.K @ E)
        r += (0.5 * sig * dt - eps) * (self.M @ E_prev) - dt * dt / (4.0 * mu) * (self.K @ E_prev)
        if F is not None:
            r += dt * dt * F
        return r

    def step(self, E: np.ndarray, E_prev: np.ndarray, F: np.ndarray | None = None) -> np.ndarray:
        """E at the next time level from the current and the previous one."""
        return self._lu.solve(self.rhs(E, E_prev, F))

    def run(self, E_prev: np.ndarray, E: np.ndarray, loads) -> list[np.ndarray]:
        """Levels E^2 .. E^{1+len(loads)} from E^0 = E_prev, E^1 = E."""
        out = []
        for F in loads:
            E_prev, E = E, self.step(E, E_prev, F)
            out.append(E)
        return out

    def energy(self, E_old: np.ndarray, E_new: np.ndarray) -> float:
        """eps/dt^2 |E_new - E_old|_M^2 + 1/(4 mu) |E_new + E_old|_K^2: constant
        from one half level to the next when sigma = 0 and F = 0, and
        non-increasing when sigma > 0 (multiply the scheme by E+ - E-)."""
        d, s = E_new - E_old, E_new + E_old
        return float(self.eps / self.dt ** 2 * (d @ (self.M @ d)) + (s @ (self.K @ s)) / (4.0 * self.mu))
