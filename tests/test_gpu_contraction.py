"""Contraction numbers of the GPU V-cycle (Sec. 5, Table 2): the error
operator E_k z = MG(k, 0, z, m) (eq. VCycleRecursion) is applied column by
column with the library's FP64 V-cycle, and ||E_k||_a is the largest
|eigenvalue| of A^{1/2} E_k A^{-1/2} (E_k is a-self-adjoint, Remark 6)."""
import os

import numpy as np
import pytest
import torch

from oracle import hcurl, mg

pytestmark = pytest.mark.gpu

try:
    from paper_2205_05840_gb300 import ndmg
except ImportError:
    if torch.cuda.is_available():
        raise
    pytest.skip("library not built and no GPU here", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))


def _table2():
    rows = {}
    with open(os.path.join(HERE, "golden", "table2_vertex.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[(float(p[0]), int(p[1]))] = [float(x) for x in p[2:]]
    return rows


def gpu_error_operator(n, alpha, m):
    """Dense E_k from the GPU V-cycle on (-1,1)^3 (L = 2, T_0 = 2^3)."""
    S = ndmg.Solver(n, n_coarsest=2, L=2.0, alpha=alpha, m=m)
    N = S.num_dofs()
    zero = torch.zeros(N, dtype=torch.float64, device="cuda")
    E = np.zeros((N, N))
    for j in range(N):
        z = torch.zeros(N, dtype=torch.float64, device="cuda")
        z[j] = 1.0
        S.vcycle(zero, z)
        torch.cuda.synchronize()
        E[:, j] = z.cpu().numpy()
    return E


def a_norm(E, A):
    Lc = np.linalg.cholesky(A)
    Sym = Lc.T @ E @ np.linalg.inv(Lc.T)
    return float(np.max(np.abs(np.linalg.eigvalsh(0.5 * (Sym + Sym.T)))))


@pytest.mark.parametrize("alpha", [0.01, 0.1, 1.0, 10.0, 100.0])
def test_table2_k1_on_gpu(alpha):
    ref = _table2()[(alpha, 1)]
    A = hcurl.assemble(4, 2.0, alpha, 1.0).toarray()
    for m in range(1, 6):
        rho = a_norm(gpu_error_operator(4, alpha, m), A)
        assert round(rho, 3) == pytest.approx(ref[m - 1], abs=1e-9), (m, rho)


@pytest.mark.parametrize("alpha,m", [(0.01, 1), (1.0, 2)])
def test_k2_contraction_matches_oracle(alpha, m):
    A = hcurl.assemble(8, 2.0, alpha, 1.0).toarray()
    rho = a_norm(gpu_error_operator(8, alpha, m), A)
    H = mg.Hierarchy(8, 2.0, alpha, 1.0, n0=2, kind="vertex", m=m)
    assert abs(rho - mg.contraction_dense(H)) < 1e-9
    assert abs(rho - _table2()[(alpha, 2)][m - 1]) < 0.03
