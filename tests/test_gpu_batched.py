"""Batched right-hand sides (nrhs > 1, right-hand side r at offset r * N):
every kernel covers the batch in one launch and the solvers iterate in
lockstep.  Each right-hand side must behave exactly like a single-RHS solve
(up to the order of atomic additions) and match the oracle."""
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


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_apply_transfer_and_dot(dtype):
    n, R = 12, 3
    S = ndmg.Solver(n, n_coarsest=3, alpha=0.4, nrhs=R)
    A = hcurl.assemble(n, 1.0, 0.4, 1.0)
    P = mg.prolongation(n // 2, 1.0)
    Nn = A.shape[0]
    X = np.random.default_rng(0).standard_normal((R, Nn))
    y = torch.empty(R * Nn, dtype=dtype, device=DEV)
    S.apply(T(X.ravel(), dtype), y)
    tol = 1e-13 if dtype == torch.float64 else 2e-6
    Xr = X.astype(np.float32).astype(np.float64) if dtype == torch.float32 else X
    for r in range(R):
        assert rel(N_(y)[r * Nn:(r + 1) * Nn], A @ Xr[r]) < tol
    gc = torch.empty(R * P.shape[1], dtype=dtype, device=DEV)
    S.restrict(T(X.ravel(), dtype), gc, level=S.num_levels - 1)
    for r in range(R):
        assert rel(N_(gc)[r * P.shape[1]:(r + 1) * P.shape[1]], P.T @ Xr[r]) < tol
    d = S.dot(T(X.ravel(), dtype), T(X.ravel(), dtype))
    for r in range(R):
        assert abs(d[r] - Xr[r] @ Xr[r]) < 1e-12 * (Xr[r] @ Xr[r]) * (1 if dtype == torch.float64 else 1e4)


@pytest.mark.parametrize("prec", [ndmg.PREC_FP64, ndmg.PREC_MIXED_BF16, ndmg.PREC_MIXED_FP16] if torch.cuda.is_available() else [0])
def test_batched_vcycle_equals_single(prec):
    n, n0, R = 16, 4, 3
    dt = torch.float64 if prec == ndmg.PREC_FP64 else torch.float32
    SB = ndmg.Solver(n, n_coarsest=n0, nrhs=R, precision=prec)
    S1 = ndmg.Solver(n, n_coarsest=n0, precision=prec)
    F = inputs.random_load(n, 5, nrhs=R)
    zb = torch.zeros(R * F.shape[1], dtype=dt, device=DEV)
    SB.vcycle(T(F.ravel(), dt), zb)
    Nn = F.shape[1]
    for r in range(R):
        z1 = torch.zeros(Nn, dtype=dt, device=DEV)
        S1.vcycle(T(F[r], dt), z1)
        # identical arithmetic per right-hand side; only the order of the
        # atomic additions differs, and in bf16/fp16 a last-bit difference can
        # flip one operand rounding (relative 2^-8 / 2^-11): allow 8 such units
        u_op = {ndmg.PREC_FP64: 1e-13 / 8, ndmg.PREC_MIXED_BF16: 2.0 ** -8, ndmg.PREC_MIXED_FP16: 2.0 ** -11}[prec]
        assert rel(N_(zb)[r * Nn:(r + 1) * Nn], N_(z1)) < 8 * u_op
    if prec == ndmg.PREC_FP64:
        H = mg.Hierarchy(n, 1.0, 1.0, 1.0, n0=n0, m=2)
        for r in range(R):
            assert rel(N_(zb)[r * Nn:(r + 1) * Nn], H.vcycle(F[r], np.zeros(Nn))) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "bf16", "fp16"])
def test_batched_solve_each_rhs_converges(prec):
    code = {"fp64": ndmg.PREC_FP64, "bf16": ndmg.PREC_MIXED_BF16, "fp16": ndmg.PREC_MIXED_FP16}[prec]
    n, n0, R = 32, 4, 4
    SB = ndmg.Solver(n, n_coarsest=n0, nrhs=R, precision=code)
    S64 = ndmg.Solver(n, n_coarsest=n0)
    F = inputs.random_load(n, 10, nrhs=R)
    F[2] *= 1e-3                                    # different scales converge at different iterations
    u = torch.zeros(F.size, dtype=torch.float64, device=DEV)
    st, it, rr = SB.solve(T(F.ravel()), u, tol=1e-8, maxit=200)
    assert rr <= 1e-8
    Nn = F.shape[1]
    for r in range(R):
        ur = u[r * Nn:(r + 1) * Nn].contiguous()
        res = torch.empty_like(ur)
        S64.residual(T(F[r]), ur, res)
        assert np.linalg.norm(N_(res)) / np.linalg.norm(F[r]) <= 1.01e-8
        u1 = torch.zeros(Nn, dtype=torch.float64, device=DEV)
        S64.solve(T(F[r]), u1, tol=1e-10)
        assert rel(N_(ur), N_(u1)) < 1e-6
    # the gradient entry point returns one value per right-hand side
    g = SB.grad_alpha(u, u)
    K, _ = hcurl.assemble_parts(n, 1.0)
    for r in range(R):
        ur = N_(u)[r * Nn:(r + 1) * Nn]
        # u^T K u of a solution cancels heavily (K has a large null space):
        # two summation orders agree to ~1e-9 relative
        assert abs(g[r] + ur @ (K @ ur)) < 1e-7 * abs(ur @ (K @ ur))


def test_batched_maxwell_steps_128():
    # 128^3, 32 right-hand sides modelling implicit Maxwell steps:
    # alpha = dt^2 / (4 mu) with dt = 1e-2, mu = 1; mass coefficient 1
    n, R = 128, 32
    alpha = 1e-2 ** 2 / 4.0
    S = ndmg.Solver(n, n_coarsest=4, alpha=alpha, nrhs=R, precision=ndmg.PREC_MIXED_FP16)
    F = np.concatenate([inputs.random_load(n, r) for r in range(R)])
    u = torch.zeros(F.size, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(T(F), u, tol=1e-8, maxit=100)
    assert rr <= 1e-8 and it < 30
    S64 = ndmg.Solver(n, n_coarsest=4, alpha=alpha)
    Nn = F.size // R
    for r in (0, 13, 31):
        ur = u[r * Nn:(r + 1) * Nn].contiguous()
        res = torch.empty_like(ur)
        S64.residual(T(F[r * Nn:(r + 1) * Nn]), ur, res)
        assert np.linalg.norm(N_(res)) / np.linalg.norm(F[r * Nn:(r + 1) * Nn]) <= 1.01e-8


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("prec", [ndmg.PREC_MIXED_BF16, ndmg.PREC_MIXED_FP16] if torch.cuda.is_available() else [0])
@pytest.mark.parametrize("n,n0,R", [(16, 4, 3), (40, 5, 2)])
def test_batched_smoothing_step_per_rhs_matches_oracle(kind, prec, n, n0, R):
    # one smoothing step z <- z + M_V^{-1}(g - A z) on a batch: every
    # right-hand side against the FP64 oracle, with the smoother kernel forced
    # (0 FP32 CUDA cores, 1 tensor-core bricks, 2 tensor-core cell rows); the
    # tensor-core kernels to 16 units of the operand rounding, the FP32 one to
    # 1e-5
    S = ndmg.Solver(n, n_coarsest=n0, nrhs=R, precision=prec)
    S.select_smoother(kind)
    A = hcurl.assemble(n, 1.0, 1.0, 1.0)
    Sm = mg.Smoother(A, n, "vertex")
    Nn = A.shape[0]
    rng = np.random.default_rng(n + R)
    G = rng.standard_normal((R, Nn)).astype(np.float32).astype(np.float64)
    Z = rng.standard_normal((R, Nn)).astype(np.float32).astype(np.float64)
    zt = T(Z.ravel(), torch.float32)
    S.smooth(T(G.ravel(), torch.float32), zt, steps=1, level=-1)
    got = N_(zt).reshape(R, Nn) - Z
    u = {ndmg.PREC_MIXED_BF16: 2.0 ** -8, ndmg.PREC_MIXED_FP16: 2.0 ** -11}[prec]
    tol = 1e-5 if kind == 0 else 16 * u
    for r in range(R):
        corr = Sm.apply(G[r] - A @ Z[r])
        assert rel(got[r], corr) < tol, (r, rel(got[r], corr))
