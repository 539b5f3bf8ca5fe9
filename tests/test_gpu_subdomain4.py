"""Subdomain size 4 (4x4x4-cell subdomains, 1176-edge vertex patches): the
GPU smoother, V-cycle and solves against the oracle's Smoother / Hierarchy
with s = 4, and the 64^3 manufactured-load configuration at s = 4."""
import numpy as np
import pytest
import torch

from oracle import hcurl, mg
from paper_2205_05840_gb300 import inputs

pytestmark = pytest.mark.gpu

try:
    from paper_2205_05840_gb300 import ndmg
except ImportError:
    if torch.cuda.is_available():
        raise
    pytest.skip("library not built and no GPU here", allow_module_level=True)

DEV = "cuda"


def T(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=DEV)


def N(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def tol4(n, alpha, base, L=1.0, beta=1.0):
    """FP64 agreement of two Cholesky-based solves with the 8x8x8-cell patch
    matrix (cond ~ alpha / (beta h^2))."""
    h = L / n
    kappa = np.linalg.cond(hcurl.assemble(8, 8 * h, alpha, beta).toarray())
    return max(base, 8.0 * kappa * np.finfo(float).eps)


@pytest.mark.parametrize("n,n0,alpha", [(8, 4, 1.0), (16, 4, 0.01), (24, 6, 100.0)])
def test_smoothing_step_parity_s4(n, n0, alpha):
    S = ndmg.Solver(n, n_coarsest=n0, alpha=alpha, subdomain=4)
    A = hcurl.assemble(n, 1.0, alpha, 1.0)
    Sm = mg.Smoother(A, n, "vertex", s=4)
    rng = np.random.default_rng(2)
    g = rng.standard_normal(A.shape[0])
    z = rng.standard_normal(A.shape[0])
    ref = z.copy()
    for _ in range(2):
        ref = ref + Sm.apply(g - A @ ref)
    zt = T(z)
    S.smooth(T(g), zt, steps=2, level=-1)
    assert rel(N(zt), ref) < tol4(n, alpha, 1e-12)
    # the float smoother of the same handle (CUDA cores at s = 4)
    z32 = T(z, torch.float32)
    S.smooth(T(g, torch.float32), z32, steps=1, level=-1)
    ref1 = z + Sm.apply(g - A @ z)
    assert rel(N(z32), ref1) < 2e-5


@pytest.mark.parametrize("n,n0,alpha,m", [(16, 4, 1.0, 2), (24, 6, 0.01, 1), (32, 4, 100.0, 2)])
def test_vcycle_iterates_parity_s4(n, n0, alpha, m):
    S = ndmg.Solver(n, n_coarsest=n0, alpha=alpha, m=m, subdomain=4)
    H = mg.Hierarchy(n, 1.0, alpha, 1.0, n0=n0, m=m, s=4)
    f = inputs.random_load(n, 0)
    z = np.zeros_like(f)
    zt, ft = T(z), T(f)
    tol = tol4(n, alpha, 1e-10)
    for it in range(4):
        z = H.vcycle(f, z)
        S.vcycle(ft, zt)
        assert rel(N(zt), z) < tol, it


def test_pcg_iterations_match_oracle_s4():
    n = 16
    S = ndmg.Solver(n, n_coarsest=4, subdomain=4)
    H = mg.Hierarchy(n, 1.0, 1.0, 1.0, n0=4, s=4)
    f = inputs.random_load(n, 1)
    u_ref, it_ref, rr_ref, _ = mg.pcg(H, f, tol=1e-8)
    u = torch.zeros(f.size, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(T(f), u, tol=1e-8)
    assert it == it_ref and rr <= 1e-8
    assert rel(N(u), u_ref) < 1e-8


@pytest.mark.parametrize("prec", [ndmg.PREC_MIXED_BF16, ndmg.PREC_MIXED_FP16, ndmg.PREC_FP32])
def test_mixed_solve_s4_reaches_fp64_tolerance(prec):
    n = 32
    S = ndmg.Solver(n, n_coarsest=4, subdomain=4, precision=prec)
    f = T(inputs.random_load(n, 2))
    u = torch.zeros_like(f)
    st, it, rr = S.solve(f, u, tol=1e-8)
    assert rr <= 1e-8
    S64 = ndmg.Solver(n, n_coarsest=4)
    r = torch.empty_like(u)
    S64.residual(f, u, r)
    assert np.linalg.norm(N(r)) <= 1.01e-8 * np.linalg.norm(N(f))


@pytest.mark.parametrize("alpha", [0.01, 1.0, 100.0])
def test_manufactured_64_s4(alpha):
    # 64^3, manufactured load, coarsest 4^3, subdomains of 4^3 cells: PCG to
    # 1e-8; the discrete solution is c * Pi u up to O(h^2)
    n = 64
    h = 1.0 / n
    S = ndmg.Solver(n, n_coarsest=4, alpha=alpha, subdomain=4)
    f = inputs.manufactured_load(n, 1.0, alpha, 1.0)
    u = torch.zeros(f.size, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(T(f), u, tol=1e-8)
    assert rr <= 1e-8 and it <= 40
    # Pi u is an exact discrete eigenvector: u_h = c Pi u in closed form
    mu = (2.0 + np.cos(np.pi * h)) / 3.0
    sig = (np.sin(np.pi * h / 2) / (np.pi * h / 2)) ** 2
    c = (2 * np.pi ** 2 * alpha + 1) * sig ** 2 / (8 * alpha * np.sin(np.pi * h / 2) ** 2 * mu / h ** 2 + mu ** 2)
    assert rel(N(u), c * inputs.sine_interpolant(n)) < 1e-6


def test_subdomain4_argument_checks():
    with pytest.raises(ndmg.NdmgError):
        ndmg.Solver(16, n_coarsest=4, subdomain=4, smoother=ndmg.SMOOTHER_EDGE)
    with pytest.raises(ndmg.NdmgError):
        ndmg.Solver(12, n_coarsest=3, subdomain=4)       # level 6 is not a multiple of 4
    with pytest.raises(ndmg.NdmgError):
        ndmg.Solver(16, n_coarsest=4, subdomain=3)
