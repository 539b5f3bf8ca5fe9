"""GPU parity for a curl-curl coefficient that is constant per hexahedron
(eq. 1 with a piecewise-constant alpha, the jumping coefficients of the
concluding remarks): field stencil, grouped local solves (CUDA cores and
tensor cores), the V-cycle and PCG, and the per-cell derivative
-lambda^T K_T u.  Every expected value comes from oracle/ (assemble_field,
Smoother(varying=True), Hierarchy with a field) on the same seeded inputs.

Tolerances: operator applications 1e-12 relative (FP64 rounding of a 33-point
stencil whose weights now spread over the field's range), FP32 2e-6; FP64
smoothing steps and V-cycle iterates 1e-10, raised to 8 cond(A_patch) eps
where the patch matrices are ill-conditioned (cond ~ max alpha / (beta h^2));
tensor-core steps 16 u of the operand precision as for a constant coefficient.
"""
import numpy as np
import pytest
import torch

from oracle import hcurl, mg
from paper_2205_05840_gb300 import inputs

pytestmark = pytest.mark.gpu

try:
    from paper_2205_05840_gb300 import autograd, ndmg
except ImportError:
    if torch.cuda.is_available():
        raise
    pytest.skip("library not built and no GPU here", allow_module_level=True)

DEV = "cuda"
U = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11}


def T(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=DEV)


def N(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def field_tol(n, a, base, L=1.0, beta=1.0):
    """8 cond eps of the worst vertex-patch matrix of the field (the patch
    with the largest coefficient bounds it), or base."""
    h = L / n
    kappa = np.linalg.cond(hcurl.assemble(4, 4 * h, float(np.max(a)), beta).toarray())
    return max(base, 8.0 * kappa * np.finfo(float).eps)


def make_field(kind, n, seed=0):
    if kind == "random":
        return inputs.random_field(n, seed, 0.1, 10.0)
    if kind == "checker":
        return inputs.checker_field(n, 2, 0.01, 100.0)
    if kind == "checker4":
        return inputs.checker_field(n, 4, 1.0, 100.0)
    return inputs.inclusion_field(n, 1.0, 100.0)


@pytest.mark.parametrize("n,n0,kind", [(4, 2, "random"), (8, 2, "random"), (12, 3, "random"), (16, 4, "random"),
                                       (40, 5, "checker"), (72, 9, "inclusion"), (36, 9, "checker4")])
def test_field_apply_and_residual(n, n0, kind):
    a = make_field(kind, n, seed=n)
    S = ndmg.Solver(n, n_coarsest=n0, beta=0.7)
    S.set_alpha_field(a)
    A = hcurl.assemble_field(n, 1.0, a, 0.7)
    rng = np.random.default_rng(n)
    x, g = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
    y = torch.empty(A.shape[0], dtype=torch.float64, device=DEV)
    S.apply(T(x), y)
    assert rel(N(y), A @ x) < 1e-12
    r = torch.empty_like(y)
    S.residual(T(g), T(x), r)
    assert rel(N(r), g - A @ x) < 1e-12
    y32 = torch.empty(A.shape[0], dtype=torch.float32, device=DEV)
    S.apply(T(x, torch.float32), y32)
    assert rel(N(y32), A @ x.astype(np.float32).astype(np.float64)) < 2e-6
    # coarser levels carry the cell means
    H = mg.Hierarchy(n, 1.0, a, 0.7, n0=n0, m=1) if n <= 16 else None
    fk = a
    for lv in range(S.num_levels - 1, -1, -1):
        nl = n0 << lv
        Al = H.A[lv] if H is not None else hcurl.assemble_field(nl, 1.0, fk, 0.7)
        xl = rng.standard_normal(Al.shape[0])
        yl = torch.empty(Al.shape[0], dtype=torch.float64, device=DEV)
        S.apply(T(xl), yl, level=lv)
        assert rel(N(yl), Al @ xl) < 1e-12, lv
        if lv > 0:
            fk = mg.coarsen_field(fk, nl)


def test_field_pencil_is_weighted_curl_curl():
    # with a field, ndmg_pencil's K is sum_T alpha_T K_T
    n = 12
    a = make_field("random", n, 3)
    S = ndmg.Solver(n, n_coarsest=3)
    S.set_alpha_field(a)
    Kf = hcurl.assemble_field(n, 1.0, a, 0.0)
    M = hcurl.assemble(n, 1.0, 0.0, 1.0)
    rng = np.random.default_rng(0)
    x, g = rng.standard_normal(Kf.shape[0]), rng.standard_normal(Kf.shape[0])
    y = torch.empty(Kf.shape[0], dtype=torch.float64, device=DEV)
    S.pencil(-0.3, 2.0, T(x), y, g=T(g))
    assert rel(N(y), g - 0.3 * (Kf @ x) + 2.0 * (M @ x)) < 1e-12


@pytest.mark.parametrize("kind,field", [("vertex", "random"), ("vertex", "checker"), ("edge", "random"),
                                        ("edge", "checker")])
def test_field_smoothing_step_fp64(kind, field):
    n = 16
    a = make_field(field, n, seed=5)
    S = ndmg.Solver(n, n_coarsest=4, smoother=ndmg.SMOOTHER_VERTEX if kind == "vertex" else ndmg.SMOOTHER_EDGE)
    S.set_alpha_field(a)
    A = hcurl.assemble_field(n, 1.0, a, 1.0)
    Sm = mg.Smoother(A, n, kind, varying=True)
    rng = np.random.default_rng(1)
    g, z = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
    zt = T(z)
    S.smooth(T(g), zt, steps=1)
    ref = z + Sm.apply(g - A @ z)
    assert rel(N(zt) - z, ref - z) < field_tol(n, a, 1e-10)


@pytest.mark.parametrize("kind,n,n0,m", [("random", 16, 2, 2), ("checker", 16, 2, 1), ("inclusion", 32, 4, 2),
                                         ("checker4", 24, 3, 2)])
def test_field_vcycle_iterates(kind, n, n0, m):
    a = make_field(kind, n, seed=7)
    H = mg.Hierarchy(n, 1.0, a, 1.0, n0=n0, m=m)
    S = ndmg.Solver(n, n_coarsest=n0, m=m)
    S.set_alpha_field(a)
    f = inputs.random_load(n, 0)
    z_ref = np.zeros_like(f)
    zt = torch.zeros(f.size, dtype=torch.float64, device=DEV)
    ft = T(f)
    tol = field_tol(n, a, 1e-10)
    for it in range(3):
        z_ref = H.vcycle(f, z_ref)
        S.vcycle(ft, zt)
        assert rel(N(zt), z_ref) < tol, it


@pytest.mark.parametrize("kind,n,n0", [("checker", 16, 2), ("inclusion", 24, 3)])
def test_field_pcg_matches_oracle(kind, n, n0):
    a = make_field(kind, n)
    H = mg.Hierarchy(n, 1.0, a, 1.0, n0=n0, m=2)
    f = inputs.random_load(n, 0)
    u_ref, it_ref, rr_ref, _ = mg.pcg(H, f, tol=1e-8)
    S = ndmg.Solver(n, n_coarsest=n0)
    S.set_alpha_field(a)
    u = torch.zeros(f.size, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(T(f), u, tol=1e-8)
    assert rr <= 1e-8 and abs(it - it_ref) <= 1
    # both solutions are within 1e-8 (relative residual) of the discrete one
    A = H.A[-1]
    kappa_bound = 1e-8 * np.linalg.norm(f)
    assert np.linalg.norm(A @ N(u) - f) <= kappa_bound * 1.0001


def test_field_interior_gradient_eigenmode():
    # curl grad psi = 0 whatever the coefficients: one V-cycle with g = 0
    # multiplies the interior gradient of a coarse-element centre hat by
    # exactly (1 - eta)^(2m)
    n, m, eta = 16, 2, 1.0 / 9.0
    a = make_field("checker", n)
    S = ndmg.Solver(n, n_coarsest=2, m=m)
    S.set_alpha_field(a)
    z0 = np.zeros(hcurl.num_edges(n))
    c = (5, 3, 9)
    for d in range(3):
        lo = list(c)
        lo[d] -= 1
        z0[hcurl.edge_index(n, d, *lo)] = 1.0
        z0[hcurl.edge_index(n, d, *c)] = -1.0
    zt = T(z0)
    S.vcycle(torch.zeros_like(zt), zt)
    assert np.abs(N(zt) - (1 - eta) ** (2 * m) * z0).max() < 1e-9


def test_constant_field_equals_scalar_coefficient():
    n = 16
    S1 = ndmg.Solver(n, n_coarsest=2, alpha=2.5)
    S2 = ndmg.Solver(n, n_coarsest=2, alpha=1.0)
    S2.set_alpha_field(np.full(n ** 3, 2.5))
    f = T(inputs.random_load(n, 3))
    z1, z2 = torch.zeros_like(f), torch.zeros_like(f)
    S1.vcycle(f, z1)
    S2.vcycle(f, z2)
    assert rel(N(z2), N(z1)) < 1e-12
    # back to a constant coefficient
    S2.set_alpha(2.5)
    z3 = torch.zeros_like(f)
    S2.vcycle(f, z3)
    assert rel(N(z3), N(z1)) < 1e-14


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("kind,n,n0", [("random", 12, 6), ("checker4", 20, 5), ("inclusion", 40, 5)])
def test_field_tc_smoothing_step(prec, kind, n, n0):
    # grouped Gram factors on tensor cores: the random field gives every patch
    # its own group (up to 80 passes per brick)
    a = make_field(kind, n, seed=2) if kind != "random" else inputs.random_field(n, 2, 0.5, 2.0)
    S = ndmg.Solver(n, n_coarsest=n0, precision=ndmg.PREC_MIXED_BF16 if prec == "bf16" else ndmg.PREC_MIXED_FP16)
    S.set_alpha_field(a)
    A = hcurl.assemble_field(n, 1.0, a, 1.0)
    Sm = mg.Smoother(A, n, "vertex", varying=True)
    rng = np.random.default_rng(n)
    g = rng.standard_normal(A.shape[0]).astype(np.float32).astype(np.float64)
    z = rng.standard_normal(A.shape[0]).astype(np.float32).astype(np.float64)
    corr = Sm.apply(g - A @ z)
    zt = T(z, torch.float32)
    S.smooth(T(g, torch.float32), zt, steps=1)
    assert rel(N(zt) - z, corr) < 16 * U[prec]


@pytest.mark.parametrize("prec", [ndmg.PREC_MIXED_BF16, ndmg.PREC_MIXED_FP16, ndmg.PREC_FP32])
@pytest.mark.parametrize("kind,n,n0", [("checker", 32, 4), ("inclusion", 64, 4)])
def test_field_mixed_solve_reaches_fp64_tolerance(prec, kind, n, n0):
    a = make_field(kind, n)
    f = T(inputs.random_load(n, 0))
    S64 = ndmg.Solver(n, n_coarsest=n0)
    S64.set_alpha_field(a)
    u64 = torch.zeros_like(f)
    _, it64, rr64 = S64.solve(f, u64, tol=1e-10, maxit=300)
    S = ndmg.Solver(n, n_coarsest=n0, precision=prec)
    if prec == ndmg.PREC_MIXED_BF16 and kind == "inclusion":
        # alpha / h^2 = 4e5 inside the inclusion: bf16 operands cannot carry
        # the patch operator (a solve diverged); the handle refuses the field
        with pytest.raises(ndmg.NdmgError) as e:
            S.set_alpha_field(a)
        assert e.value.status == ndmg.INVALID_ARG
        return
    S.set_alpha_field(a)
    u = torch.zeros_like(f)
    st, it, rr = S.solve(f, u, tol=1e-8, maxit=300)
    assert rr <= 1e-8
    # the low-precision preconditioner costs at most a few more iterations
    assert it <= 3 * it64 + 10
    # the residual, recomputed with the oracle's operator
    A = hcurl.assemble_field(n, 1.0, a, 1.0)
    fh = N(f)
    assert np.linalg.norm(fh - A @ N(u)) <= 1.01e-8 * np.linalg.norm(fh)


@pytest.mark.parametrize("n", [6, 8, 12])
def test_grad_cells_matches_oracle_elements(n):
    rng = np.random.default_rng(n)
    Nn = hcurl.num_edges(n)
    lam, u = rng.standard_normal((2, Nn))
    R = 2
    S = ndmg.Solver(n, n_coarsest=n // 2 if n % 4 else n // 4, nrhs=R)
    lamR = np.concatenate([lam, 2.0 * lam])
    uR = np.concatenate([u, -u])
    got = N(S.grad_alpha_field(T(lamR), T(uR)))
    KT, _ = hcurl.element_matrices(1.0 / n)
    dofs = hcurl._element_dofs(n)
    ln = np.where(dofs >= 0, lam[np.maximum(dofs, 0)], 0.0)
    un = np.where(dofs >= 0, u[np.maximum(dofs, 0)], 0.0)
    ref = -np.einsum("ca,ab,cb->c", ln, KT, un)
    assert got.shape == (R * n ** 3,)
    assert rel(got[:n ** 3], ref) < 1e-13
    assert rel(got[n ** 3:], -2.0 * ref) < 1e-13
    # summed with the field's weights they give -lambda^T K_alpha u
    a = make_field("random", n, 1)
    K = hcurl.assemble_field(n, 1.0, a, 0.0)
    assert abs(a @ ref + lam @ (K @ u)) < 1e-12 * abs(lam) @ abs(K @ u)


def test_grad_field_finite_differences():
    # L = 0.5 ||u(alpha) - u_t||^2, A(alpha) u = f: dL/dalpha_T = -lambda^T K_T u
    # with A lambda = u - u_t, against the oracle's direct-solve gradient per
    # cell and against central differences along a direction that moves every
    # cell (a single cell moves u too little for the solve tolerance)
    n = 8
    a = make_field("random", n, 4)
    f_np = inputs.random_load(n, 0)
    ut = inputs.random_target(n, 1) * 0.05
    f = T(f_np)
    S = ndmg.Solver(n, n_coarsest=2)

    def solve(field):
        S.set_alpha_field(field)
        u = torch.zeros_like(f)
        S.solve(f, u, tol=1e-13, maxit=400)
        return u

    u = solve(a)
    lam = torch.zeros_like(u)
    S.solve(T(N(u) - ut), lam, tol=1e-13, maxit=400)
    grad = N(S.grad_alpha_field(lam, u))
    _, g_ref, _ = mg.loss_and_grad_field(n, 1.0, a, 1.0, f_np, ut)
    assert rel(grad, g_ref) < 1e-7
    d = np.random.default_rng(9).choice([-1.0, 1.0], n ** 3) * a
    eps = 1e-4
    Lp = 0.5 * np.sum((N(solve(a + eps * d)) - ut) ** 2)
    Lm = 0.5 * np.sum((N(solve(a - eps * d)) - ut) ** 2)
    fd = (Lp - Lm) / (2 * eps)
    assert abs(fd - grad @ d) <= 1e-5 * abs(fd)


def test_field_rejects_bad_input_and_keeps_working():
    n = 64
    S = ndmg.Solver(n, n_coarsest=4)
    f = T(inputs.random_load(n, 0))
    u0 = torch.zeros_like(f)
    S.solve(f, u0, tol=1e-8)
    with pytest.raises(ndmg.NdmgError) as e:
        S.set_alpha_field(inputs.random_field(n, 0))      # 29,791 distinct vertex patches > 8192
    assert e.value.status == ndmg.INVALID_ARG
    bad = np.ones(n ** 3)
    bad[5] = -1.0
    with pytest.raises(ndmg.NdmgError):
        S.set_alpha_field(bad)
    bad[5] = np.nan
    with pytest.raises(ndmg.NdmgError):
        S.set_alpha_field(bad)
    u = torch.zeros_like(f)
    st, it, rr = S.solve(f, u, tol=1e-8)
    assert rr <= 1e-8 and rel(N(u), N(u0)) < 1e-12
    S4 = ndmg.Solver(16, n_coarsest=4, subdomain=4)
    with pytest.raises(ndmg.NdmgError):
        S4.set_alpha_field(np.ones(16 ** 3))


def test_autograd_field_gradient():
    # torch autograd over the field solve: dL/df = lambda and dL/dalpha_T =
    # -lambda^T K_T u, against central differences of the loss
    n = 8
    a0 = make_field("random", n, 6)
    S = ndmg.Solver(n, n_coarsest=2)
    f = torch.tensor(inputs.random_load(n, 0), device=DEV, requires_grad=True)
    ut = torch.tensor(0.05 * inputs.random_target(n, 1), device=DEV)
    a = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    u = autograd.solve_field(f, a, S, tol=1e-13)
    loss = 0.5 * ((u - ut) ** 2).sum()
    loss.backward()
    ga = a.grad.numpy()
    gf = f.grad.detach().cpu().numpy()

    def L_of(field, load):
        with torch.no_grad():
            uu = autograd.solve_field(load, torch.tensor(field), S, tol=1e-13)
            return float(0.5 * ((uu - ut) ** 2).sum())

    dd = np.random.default_rng(2).choice([-1.0, 1.0], n ** 3) * a0
    eps = 1e-4
    fd = (L_of(a0 + eps * dd, f.detach()) - L_of(a0 - eps * dd, f.detach())) / (2 * eps)
    assert abs(fd - ga @ dd) <= 1e-5 * abs(fd)
    rng = np.random.default_rng(0)
    d = torch.tensor(rng.standard_normal(f.numel()), device=DEV)
    eps = 1e-3
    fd = (L_of(a0, f.detach() + eps * d) - L_of(a0, f.detach() - eps * d)) / (2 * eps)
    assert abs(fd - gf @ d.cpu().numpy()) <= 1e-6 * abs(fd)
