"""Host-side fault injection and large-batch launch limits, through the C ABI.

The device status word is what a tensor-core kernel sets when one of its
bounded mbarrier waits gives up.  No GPU test makes such a wait run out (a
forced timeout would leave tensor-core work in flight); instead the word is
set from the host (ndmg_inject_status) and the tests check that the next
solve reports NDMG_DEVICE_TIMEOUT, clears it, and that the handle then solves
as before."""
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


@pytest.mark.parametrize("prec", [ndmg.PREC_MIXED_FP16, ndmg.PREC_MIXED_BF16])
def test_injected_timeout_is_reported_and_cleared(prec):
    n = 16
    S = ndmg.Solver(n, n_coarsest=4, precision=prec)
    f = torch.tensor(inputs.random_load(n, 0), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    st, it, rr = S.solve(f, u, tol=1e-8)
    assert st == ndmg.OK and rr <= 1e-8
    u_ok = u.clone()
    # a solve after the word was set reports the timeout
    S.inject_status(1)
    u.zero_()
    with pytest.raises(ndmg.NdmgError) as ei:
        S.solve(f, u, tol=1e-8)
    assert ei.value.status == ndmg.DEVICE_TIMEOUT
    # ... and cleared it: the handle solves as before
    u.zero_()
    st, it2, rr2 = S.solve(f, u, tol=1e-8)
    assert st == ndmg.OK and rr2 <= 1e-8 and it2 == it
    assert torch.allclose(u, u_ok, rtol=0, atol=1e-6 * float(u_ok.abs().max()))
    # the float V-cycle entry point reads the word too
    g32 = f.float()
    z32 = torch.zeros_like(g32)
    S.inject_status(3)
    with pytest.raises(ndmg.NdmgError) as ei:
        S.vcycle(g32, z32)
    assert ei.value.status == ndmg.DEVICE_TIMEOUT
    z32.zero_()
    S.vcycle(g32, z32)
    assert torch.isfinite(z32).all() and float(z32.abs().max()) > 0


def test_batched_gradient_sums_over_right_hand_sides():
    # a batch shares alpha: dL/dalpha of sum_r L_r is the sum of the
    # per-right-hand-side -lambda_r^T K u_r; compared with the oracle's adjoint
    # gradient of each right-hand side
    n, R, alpha0 = 16, 2, 0.7
    S = ndmg.Solver(n, n_coarsest=4, alpha=alpha0, nrhs=R)
    fs = [inputs.random_load(n, s) for s in range(R)]
    uts = [1e-3 * inputs.random_target(n, 10 + s) for s in range(R)]
    f = torch.tensor(np.concatenate(fs), device="cuda", requires_grad=True)
    ut = torch.tensor(np.concatenate(uts), device="cuda")
    alpha = torch.tensor(alpha0, dtype=torch.float64, requires_grad=True)
    u = autograd.solve(f, alpha, S, tol=1e-11)
    loss = 0.5 * ((u - ut) ** 2).sum()
    loss.backward()
    H = mg.Hierarchy(n, 1.0, alpha0, 1.0, n0=4, m=2)
    ref = 0.0
    for fr, utr in zip(fs, uts):
        _, _, da, _ = mg.loss_and_grad(H, fr, utr, tol=1e-11)
        ref += da
    assert alpha.grad.shape == alpha.shape
    assert abs(float(alpha.grad) - ref) < 1e-6 * abs(ref)


@pytest.mark.parametrize("op", ["restrict", "prolong"])
def test_transfers_with_more_planes_times_rhs_than_grid_z(op):
    # coarse planes x right-hand sides above the 65,535 limit of grid z: the
    # launcher splits the batch.  36^3 -> 18^3 with 3,641 right-hand sides
    # (18 x 3,641 = 65,538); a handful of right-hand sides, including both
    # sides of the split, against the oracle's transfer matrix
    nf, nc, R = 36, 18, 3641
    need = 50e9
    if torch.cuda.mem_get_info()[0] < need:
        pytest.skip("not enough free device memory for the 3,641-right-hand-side handle")
    S = ndmg.Solver(nf, n_coarsest=9, precision=ndmg.PREC_FP32, nrhs=R)
    Nf, Nc = S.num_dofs(-1), S.num_dofs(S.num_levels - 2)
    gen = torch.Generator(device="cuda").manual_seed(7)
    P = mg.prolongation(nc, 1.0)
    check = [0, 1, 65535 // nc - 1, 65535 // nc, R - 1]
    if op == "restrict":
        x = torch.rand(Nf * R, generator=gen, device="cuda", dtype=torch.float32) * 2 - 1
        y = torch.full((Nc * R,), float("nan"), device="cuda", dtype=torch.float32)
        S.restrict(x, y, level=-1)
        torch.cuda.synchronize()
        for r in check:
            xr = x[r * Nf:(r + 1) * Nf].double().cpu().numpy()
            yr = y[r * Nc:(r + 1) * Nc].double().cpu().numpy()
            ref = P.T @ xr
            assert np.abs(yr - ref).max() <= 2e-6 * np.abs(ref).max(), r
    else:
        x = torch.rand(Nc * R, generator=gen, device="cuda", dtype=torch.float32) * 2 - 1
        y0 = torch.rand(Nf * R, generator=gen, device="cuda", dtype=torch.float32)
        y = y0.clone()
        S.prolong_add(x, y, level=-1)
        torch.cuda.synchronize()
        for r in check:
            xr = x[r * Nc:(r + 1) * Nc].double().cpu().numpy()
            ref = y0[r * Nf:(r + 1) * Nf].double().cpu().numpy() + P @ xr
            yr = y[r * Nf:(r + 1) * Nf].double().cpu().numpy()
            assert np.abs(yr - ref).max() <= 2e-6 * np.abs(ref).max(), r
    del S, x, y
    torch.cuda.empty_cache()
