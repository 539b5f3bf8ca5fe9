"""Implicit Maxwell time stepping on the GPU (Sec. 1, eq. (Maxwell timestep))
against the FP64 oracle's stepper (direct solves), the closed-form evolution
of an exact eigenmode, and the pencil / vector-update entry points against
the oracle's K and M."""
import numpy as np
import pytest
import torch

from oracle import hcurl, maxwell as omax
from paper_2205_05840_gb300 import inputs

pytestmark = pytest.mark.gpu

try:
    from paper_2205_05840_gb300 import maxwell, ndmg
except ImportError:
    if torch.cuda.is_available():
        raise
    pytest.skip("library not built and no GPU here", allow_module_level=True)

DEV = "cuda"


def T(a, dt=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dt, device=DEV)


def N_(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n,n0,R", [(12, 3, 1), (40, 5, 1), (16, 4, 3)])
def test_pencil_and_axpby_parity(n, n0, R):
    S = ndmg.Solver(n, n_coarsest=n0, L=1.5, alpha=0.3, nrhs=R)
    K, M = hcurl.assemble_parts(n, 1.5)
    Nn = K.shape[0]
    rng = np.random.default_rng(n)
    x, g = rng.standard_normal((2, R * Nn))
    a, b = -0.37, 2.1
    ref = np.concatenate([g[r * Nn:(r + 1) * Nn] + a * (K @ x[r * Nn:(r + 1) * Nn]) + b * (M @ x[r * Nn:(r + 1) * Nn])
                          for r in range(R)])
    y = T(g)                                   # y aliases g
    S.pencil(a, b, T(x), y, g=y)
    assert rel(N_(y), ref) < 1e-13
    y2 = torch.empty(R * Nn, dtype=torch.float64, device=DEV)
    S.pencil(a, b, T(x), y2)
    assert rel(N_(y2), ref - g) < 1e-13
    # FP32 vectors: same pencil in float arithmetic
    y3 = torch.empty(R * Nn, dtype=torch.float32, device=DEV)
    S.pencil(a, b, T(x, torch.float32), y3, g=T(g, torch.float32))
    assert rel(N_(y3), ref) < 5e-6
    z = T(g)
    S.axpby(2.5, T(x), -0.5, z)
    assert np.abs(N_(z) - (2.5 * x - 0.5 * g)).max() < 1e-15 * 4
    w = torch.full((R * Nn,), float("nan"), dtype=torch.float64, device=DEV)
    S.axpby(3.0, T(x), 0.0, w)                  # b = 0 does not read y
    assert np.array_equal(N_(w), 3.0 * x)
    with pytest.raises(ndmg.NdmgError):
        xx = T(x)
        S.pencil(a, b, xx, xx)


@pytest.mark.parametrize("prec", [ndmg.PREC_FP64, ndmg.PREC_MIXED_FP16])
def test_time_steps_match_oracle(prec):
    n, dt, eps, sigma, mu = 16, 0.05, 1.2, 0.4, 0.9
    ref = omax.ImplicitMaxwell(n, 1.0, dt, eps, sigma, mu)
    Nn = hcurl.num_edges(n)
    rng = np.random.default_rng(11)
    E0, E1 = rng.standard_normal((2, Nn))
    loads = [inputs.random_load(n, 20 + s) for s in range(5)]
    want = ref.run(E0, E1, loads)
    drv = maxwell.ImplicitMaxwell(n, dt, eps, sigma, mu, n_coarsest=4, precision=prec, tol=1e-12)
    got = drv.run(T(E0), T(E1), [T(F) for F in loads])
    for s, (g, w) in enumerate(zip(got, want)):
        assert rel(N_(g), w) < 1e-9, s
    # warm starts: later steps need no more iterations than the first
    assert max(drv.iterations[1:]) <= drv.iterations[0] + 1


def test_eigenmode_closed_form_on_gpu():
    # the exact eigenmode phi (K phi = lam M phi) evolves as cos(n theta) phi
    n, dt, eps, mu = 32, 0.02, 1.0, 1.0
    h = 1.0 / n
    lam = 8 * np.sin(np.pi * h / 2) ** 2 / (h * h * (2 + np.cos(np.pi * h)) / 3)
    a, b = eps / dt ** 2, lam / (4 * mu)
    theta = np.arccos((a - b) / (a + b))
    phi = inputs.sine_interpolant(n)
    drv = maxwell.ImplicitMaxwell(n, dt, eps, 0.0, mu, n_coarsest=4, precision=ndmg.PREC_MIXED_FP16, tol=1e-12)
    Es = drv.run(T(phi), T(np.cos(theta) * phi), [None] * 12)
    for s, E in enumerate(Es, start=2):
        assert np.abs(N_(E) - np.cos(s * theta) * phi).max() < 1e-9


def test_batched_fields_step_together():
    # 4 fields with different sources through the batched path, each equal
    # to its own single-field FP64 run
    n, R, dt = 32, 4, 0.01
    Nn = hcurl.num_edges(n)
    rng = np.random.default_rng(5)
    E0, E1 = rng.standard_normal((2, R * Nn))
    loads = [np.concatenate([inputs.random_load(n, 100 * s + r) for r in range(R)]) for s in range(3)]
    drv = maxwell.ImplicitMaxwell(n, dt, sigma=0.2, nrhs=R, precision=ndmg.PREC_MIXED_FP16, tol=1e-10)
    got = drv.run(T(E0), T(E1), [T(F) for F in loads])
    one = maxwell.ImplicitMaxwell(n, dt, sigma=0.2, nrhs=1, precision=ndmg.PREC_FP64, tol=1e-10)
    for r in (0, 3):
        sl = slice(r * Nn, (r + 1) * Nn)
        ref = one.run(T(E0[sl]), T(E1[sl]), [T(F[sl]) for F in loads])
        for g, w in zip(got, ref):
            assert rel(N_(g)[sl], N_(w)) < 1e-8
