"""Run-to-run agreement and read-before-write detection, through the C ABI.

The smoothers add overlapping patch contributions with atomics, so the order
of those additions (and with it the last bits of a result) may change from
run to run; everything else is deterministic.  Two solves of the same problem
must therefore take the same number of iterations and agree to a bound set by
the arithmetic: FP64 to a few units of 1e-16 per V-cycle, propagated through
the solve; the float V-cycle to its own rounding, damped by the FP64 PCG.

A handle created with NDMG_POISON_WORKSPACES=1 starts every workspace as NaN
bit patterns: any read of an entry no kernel has written would make the
solve NaN, so its results must equal those of an ordinary handle."""
import os

import numpy as np
import pytest
import torch

from paper_2205_05840_gb300 import inputs

pytestmark = pytest.mark.gpu

try:
    from paper_2205_05840_gb300 import ndmg
except ImportError:
    if torch.cuda.is_available():
        raise
    pytest.skip("library not built and no GPU here", allow_module_level=True)


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


PRECS = {"fp64": (ndmg.PREC_FP64, 1e-11), "fp16": (ndmg.PREC_MIXED_FP16, 1e-6), "bf16": (ndmg.PREC_MIXED_BF16, 1e-6)}
# one float V-cycle: a last-bit change of an FP32 sum can flip the rounding of
# a bf16 / fp16 operand (relative 2^-8 / 2^-11); allow 8 such units
CYCLE = {"fp64": 1e-13, "fp16": 8 * 2.0 ** -11, "bf16": 8 * 2.0 ** -8}


@pytest.mark.parametrize("prec", list(PRECS))
def test_two_runs_agree(prec):
    code, bound = PRECS[prec]
    n = 32
    S = ndmg.Solver(n, n_coarsest=4, precision=code)
    f = torch.tensor(inputs.random_load(n, 3), dtype=torch.float64, device="cuda")
    u1, u2 = torch.zeros_like(f), torch.zeros_like(f)
    _, it1, rr1 = S.solve(f, u1, tol=1e-8)
    _, it2, rr2 = S.solve(f, u2, tol=1e-8)
    assert it1 == it2 and rr1 <= 1e-8 and rr2 <= 1e-8
    assert rel(u2, u1) < bound
    # one V-cycle twice: same bound per cycle
    dt = torch.float64 if code == ndmg.PREC_FP64 else torch.float32
    g = f.to(dt)
    z1, z2 = torch.zeros_like(g), torch.zeros_like(g)
    S.vcycle(g, z1)
    S.vcycle(g, z2)
    assert rel(z2, z1) < CYCLE[prec]


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("nrhs", [1, 2])
def test_poisoned_workspaces_change_nothing(prec, nrhs, monkeypatch):
    code, bound = PRECS[prec]
    n = 32
    F = inputs.random_load(n, 4, nrhs=nrhs) if nrhs > 1 else inputs.random_load(n, 4)[None, :]
    f = torch.tensor(F.ravel(), dtype=torch.float64, device="cuda")
    S0 = ndmg.Solver(n, n_coarsest=4, precision=code, nrhs=nrhs)
    u0 = torch.zeros_like(f)
    _, it0, _ = S0.solve(f, u0, tol=1e-8)
    monkeypatch.setenv("NDMG_POISON_WORKSPACES", "1")
    S1 = ndmg.Solver(n, n_coarsest=4, precision=code, nrhs=nrhs)
    monkeypatch.delenv("NDMG_POISON_WORKSPACES")
    u1 = torch.zeros_like(f)
    st, it1, rr1 = S1.solve(f, u1, tol=1e-8)
    assert torch.isfinite(u1).all()
    assert st == ndmg.OK and it1 == it0 and rr1 <= 1e-8
    assert rel(u1, u0) < bound
    # the other entry points on a fresh poisoned handle
    monkeypatch.setenv("NDMG_POISON_WORKSPACES", "1")
    S2 = ndmg.Solver(n, n_coarsest=4, precision=code, nrhs=nrhs)
    monkeypatch.delenv("NDMG_POISON_WORKSPACES")
    dt = torch.float64 if code == ndmg.PREC_FP64 else torch.float32
    g = f.to(dt)
    za, zb = torch.zeros_like(g), torch.zeros_like(g)
    S0.vcycle(g, za)
    S2.vcycle(g, zb)
    assert torch.isfinite(zb).all() and rel(zb, za) < CYCLE[prec]
    y = torch.empty_like(g)
    S2.smooth(g, y.zero_(), steps=2)
    assert torch.isfinite(y).all()
    assert os.environ.get("NDMG_POISON_WORKSPACES") is None
