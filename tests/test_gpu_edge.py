"""The edge-based smoother of eq. (Preconditioner E) (eta_E = 1/13) on the
GPU against the FP64 oracle: one smoothing step, V-cycle iterates, the
interior gradient eigenmode, and a preconditioned solve.  (Parity against the
paper's Table 1 is unpinned; the oracle's own pins are its invariants.)"""
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


def N_(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("n,n0,alpha", [(4, 2, 1.0), (8, 4, 0.3), (12, 6, 3.0)])
def test_edge_smoothing_step(n, n0, alpha):
    S = ndmg.Solver(n, n_coarsest=n0, alpha=alpha, smoother=ndmg.SMOOTHER_EDGE)
    A = hcurl.assemble(n, 1.0, alpha, 1.0)
    Sm = mg.Smoother(A, n, "edge")
    rng = np.random.default_rng(n)
    g, z = rng.standard_normal((2, A.shape[0]))
    ref = z + Sm.apply(g - A @ z)
    zt = T(z)
    S.smooth(T(g), zt, steps=1)
    assert rel(N_(zt), ref) < 1e-12
    # float vectors: same operator in FP32
    z32 = T(z, torch.float32)
    S.smooth(T(g, torch.float32), z32, steps=1)
    assert rel(N_(z32), ref) < 1e-4


@pytest.mark.parametrize("n,n0,m", [(8, 2, 2), (16, 4, 1)])
def test_edge_vcycle_iterates(n, n0, m):
    S = ndmg.Solver(n, n_coarsest=n0, smoother=ndmg.SMOOTHER_EDGE, m=m)
    H = mg.Hierarchy(n, 1.0, 1.0, 1.0, n0=n0, kind="edge", m=m)
    f = inputs.random_load(n, 1)
    z = np.zeros_like(f)
    zt = torch.zeros(f.size, dtype=torch.float64, device=DEV)
    for _ in range(4):
        z = H.vcycle(f, z)
        S.vcycle(T(f), zt)
        assert rel(N_(zt), z) < 1e-10


def test_edge_interior_eigenmode():
    # grad of the fine hat at a coarse element centre: one V-cycle with g = 0
    # multiplies it by (1 - 1/13)^(2m) (it is a-orthogonal to every edge space)
    n, m = 8, 2
    S = ndmg.Solver(n, n_coarsest=2, smoother=ndmg.SMOOTHER_EDGE, m=m)
    z0 = np.zeros(hcurl.num_edges(n))
    c = (3, 1, 5)
    for d in range(3):
        lo = list(c)
        lo[d] -= 1
        z0[hcurl.edge_index(n, d, *lo)] = n
        z0[hcurl.edge_index(n, d, *c)] = -n
    zt = T(z0)
    S.vcycle(torch.zeros_like(zt), zt)
    assert rel(N_(zt), (12 / 13) ** (2 * m) * z0) < 1e-12


@pytest.mark.parametrize("prec", [0, 3])
def test_edge_preconditioned_solve(prec):
    n = 32
    S = ndmg.Solver(n, n_coarsest=4, smoother=ndmg.SMOOTHER_EDGE, precision=prec)
    f = inputs.random_load(n, 2)
    u = torch.zeros(f.size, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(T(f), u, tol=1e-8, maxit=400)
    assert rr <= 1e-8
    S64 = ndmg.Solver(n, n_coarsest=4)
    u64 = torch.zeros_like(u)
    S64.solve(T(f), u64, tol=1e-10)
    assert rel(N_(u), N_(u64)) < 1e-6
