"""Pins of the implicit Maxwell time-stepping oracle (Sec. 1, eq. (Maxwell
timestep)) against facts that do not come from its own code: the discrete
dispersion relation of an exact eigenmode (closed form) and the discrete
energy identity obtained by multiplying the scheme by E+ - E-."""
import numpy as np
import pytest

from oracle import hcurl, maxwell
from paper_2205_05840_gb300 import inputs


def test_step_operator_is_the_model_problem():
    # alpha = dt^2 / (4 mu), beta = eps + sigma dt / 2 (eq. (Maxwell timestep))
    S = maxwell.ImplicitMaxwell(4, 1.0, dt=0.1, eps=2.0, sigma=3.0, mu=0.5)
    A = hcurl.assemble(4, 1.0, 0.1 ** 2 / 2.0, 2.0 + 0.15)
    assert abs(S.A - A).max() < 1e-15 * abs(A).max()


@pytest.mark.parametrize("n,dt,eps,mu", [(6, 0.05, 1.0, 2.0), (8, 0.3, 0.5, 1.0)])
def test_eigenmode_follows_discrete_dispersion(n, dt, eps, mu):
    # the sine field phi is an exact generalised eigenvector, K phi = lam M phi
    # with lam = 8 sin^2(pi h / 2) / (h^2 (2 + cos pi h) / 3); a mode started
    # with E^0 = phi, E^1 = cos(theta) phi stays cos(n theta) phi, where
    # cos(theta) = (eps/dt^2 - lam/(4 mu)) / (eps/dt^2 + lam/(4 mu))
    h = 1.0 / n
    phi = inputs.sine_interpolant(n)
    lam = 8 * np.sin(np.pi * h / 2) ** 2 / (h * h * (2 + np.cos(np.pi * h)) / 3)
    a, b = eps / dt ** 2, lam / (4 * mu)
    theta = np.arccos((a - b) / (a + b))
    S = maxwell.ImplicitMaxwell(n, 1.0, dt=dt, eps=eps, sigma=0.0, mu=mu)
    Es = S.run(phi, np.cos(theta) * phi, [None] * 20)
    for step, E in enumerate(Es, start=2):
        assert np.allclose(E, np.cos(step * theta) * phi, rtol=0, atol=1e-11)


@pytest.mark.parametrize("sigma,with_load", [(0.0, False), (0.7, False), (0.7, True)])
def test_discrete_energy_identity(sigma, with_load):
    # W^{n+1/2} - W^{n-1/2} + sigma/(2 dt) |E+ - E-|_M^2 = F . (E+ - E-)
    n, dt = 6, 0.2
    S = maxwell.ImplicitMaxwell(n, 1.0, dt=dt, eps=1.3, sigma=sigma, mu=0.8)
    rng = np.random.default_rng(4)
    N = hcurl.num_edges(n)
    E_prev, E = rng.standard_normal(N), rng.standard_normal(N)
    for _ in range(8):
        F = rng.standard_normal(N) if with_load else None
        E_new = S.step(E, E_prev, F)
        lhs = S.energy(E, E_new) - S.energy(E_prev, E)
        d = E_new - E_prev
        lhs += sigma / (2 * dt) * (d @ (S.M @ d))
        rhs = (F @ d) if with_load else 0.0
        assert abs(lhs - rhs) < 1e-11 * S.energy(E, E_new)
        if sigma > 0 and not with_load:
            assert S.energy(E, E_new) < S.energy(E_prev, E)
        E_prev, E = E, E_new
