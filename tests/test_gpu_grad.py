"""Differentiable solve: autograd backward = adjoint solve with the same
V-cycle, dL/dalpha = -lambda^T K u (fused stencil + FP64 reduction), checked
against the FP64 oracle's adjoint gradient and central finite differences at
32^3 (loss 0.5 ||u(f, alpha) - u_t||^2)."""
import numpy as np
import pytest
import torch

from oracle import mg
from paper_2205_05840_gb300 import inputs

pytestmark = pytest.mark.gpu

try:
    from paper_2205_05840_gb300 import autograd, ndmg
except ImportError:
    if torch.cuda.is_available():
        raise
    pytest.skip("library not built and no GPU here", allow_module_level=True)


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_gradient_matches_oracle_and_fd(prec):
    n, alpha0 = 32, 0.7
    code = {"fp64": ndmg.PREC_FP64, "bf16": ndmg.PREC_MIXED_BF16}[prec]
    S = ndmg.Solver(n, n_coarsest=4, alpha=alpha0, precision=code)
    f_np = inputs.random_load(n, 0)
    ut_np = 1e-3 * inputs.random_target(n, 1)
    f = torch.tensor(f_np, device="cuda", requires_grad=True)
    alpha = torch.tensor(alpha0, dtype=torch.float64, requires_grad=True)
    ut = torch.tensor(ut_np, device="cuda")
    u = autograd.solve(f, alpha, S, tol=1e-10)
    loss = 0.5 * ((u - ut) ** 2).sum()
    loss.backward()
    g_alpha = float(alpha.grad)
    g_f = f.grad.detach().cpu().numpy()

    H = mg.Hierarchy(n, 1.0, alpha0, 1.0, n0=4, m=2)
    L_ref, lam_ref, dalpha_ref, _ = mg.loss_and_grad(H, f_np, ut_np, tol=1e-10)
    assert abs(float(loss) - L_ref) < 1e-7 * L_ref
    assert abs(g_alpha - dalpha_ref) < 1e-5 * abs(dalpha_ref)
    assert np.abs(g_f - lam_ref).max() < 1e-5 * np.abs(lam_ref).max()

    # the finite-difference losses need solves well below the difference
    # they resolve (the FP64 outer iteration reaches 1e-12 in either mode)
    def L(a):
        with torch.no_grad():
            uu = autograd.solve(f.detach(), torch.tensor(a, dtype=torch.float64), S, tol=1e-12)
            return 0.5 * float(((uu - ut) ** 2).sum())
    eps = 1e-4 * alpha0
    fd = (L(alpha0 + eps) - L(alpha0 - eps)) / (2 * eps)
    assert abs(g_alpha - fd) < 1e-5 * abs(fd)
    # f-direction derivative along a random direction
    v = torch.tensor(np.random.default_rng(2).standard_normal(f_np.size), device="cuda")
    t = 1e-3
    with torch.no_grad():
        Lp = 0.5 * float(((autograd.solve(f.detach() + t * v, torch.tensor(alpha0, dtype=torch.float64), S, 1e-12) - ut) ** 2).sum())
        Lm = 0.5 * float(((autograd.solve(f.detach() - t * v, torch.tensor(alpha0, dtype=torch.float64), S, 1e-12) - ut) ** 2).sum())
    fdf = (Lp - Lm) / (2 * t)
    assert abs(float((f.grad * v).sum()) - fdf) < 1e-5 * abs(fdf)


def test_gradient_96_cubed_directional_fd():
    # the differentiable-solve configuration: 96^3 (coarsest 3^3), loss
    # 0.5 ||u(f, alpha) - u_t||^2 with u_t from seed 1; the adjoint gradient
    # agrees with central differences along alpha and along a random f-direction
    n, alpha0 = 96, 1.0
    S = ndmg.Solver(n, n_coarsest=3, alpha=alpha0, precision=ndmg.PREC_MIXED_BF16)
    f = torch.tensor(inputs.random_load(n, 0), device="cuda", requires_grad=True)
    ut = torch.tensor(1e-3 * inputs.random_target(n, 1), device="cuda")
    a = torch.tensor(alpha0, dtype=torch.float64, requires_grad=True)
    u = autograd.solve(f, a, S, tol=1e-10)
    loss = 0.5 * ((u - ut) ** 2).sum()
    loss.backward()

    def L(al, ff):
        with torch.no_grad():
            uu = autograd.solve(ff, torch.tensor(al, dtype=torch.float64), S, tol=1e-12)
            return 0.5 * float(((uu - ut) ** 2).sum())
    eps = 1e-4 * alpha0
    fd = (L(alpha0 + eps, f.detach()) - L(alpha0 - eps, f.detach())) / (2 * eps)
    assert abs(float(a.grad) - fd) < 1e-5 * abs(fd)
    v = torch.tensor(np.random.default_rng(3).standard_normal(f.numel()), device="cuda")
    t = 1e-3
    fdf = (L(alpha0, f.detach() + t * v) - L(alpha0, f.detach() - t * v)) / (2 * t)
    assert abs(float((f.grad * v).sum()) - fdf) < 1e-5 * abs(fdf)
