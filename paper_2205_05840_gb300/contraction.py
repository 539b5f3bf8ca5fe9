"""Contraction numbers of the V-cycle on the GPU (Sec. 5, Tables 1 and 2).

The contraction number of level k is read as ||E_k||_a, the a-norm of the
error operator E_k z = MG(k, 0, z, m) (eq. VCycleRecursion).  E_k is
a-self-adjoint and a-positive semidefinite (Remark 6), so the Lanczos process
in the inner product (x, y)_a = x^T A_k y gives Ritz values that approach
||E_k||_a from below.  Each Lanczos step is one library V-cycle (the error
propagation: right-hand side 0, initial guess v) and one library operator
apply; the Krylov basis (a few hundred vectors of at most a few hundred
thousand entries) and its reorthogonalisation stay in device tensors.

    python -m paper_2205_05840_gb300.contraction --k 1 2 3 4 --alpha 0.01 1 100

prints the rows of Table 2 (vertex smoother, eta = 1/9, Omega = (-1,1)^3,
T_0 = 2^3, level k has 2^(k+1) cells per side) or, with --smoother edge, of
Table 1 (eta = 1/13).
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import ndmg


def contraction(n: int, alpha: float, m: int, *, L: float = 2.0, beta: float = 1.0, n_coarsest: int = 2,
                smoother: int = ndmg.SMOOTHER_VERTEX, steps: int = 150, z0: np.ndarray | None = None,
                seed: int = 0, solver: ndmg.Solver | None = None) -> float:
    """||E_k||_a on an n^3 grid of the cube of side L (FP64 V-cycle).

    z0 is the Lanczos start vector (seeded standard normal when omitted); the
    process stops after `steps` steps or when the Krylov space is exhausted."""
    S = solver if solver is not None else ndmg.Solver(n, n_coarsest=n_coarsest, L=L, alpha=alpha, beta=beta,
                                                      smoother=smoother, m=m)
    N = S.num_dofs()
    dev = torch.device("cuda")
    if z0 is None:
        z0 = np.random.default_rng(seed).standard_normal(N)
    steps = min(steps, N)
    V = torch.zeros(steps, N, dtype=torch.float64, device=dev)   # a-orthonormal basis
    AV = torch.zeros_like(V)                                      # A_k times the basis
    zero = torch.zeros(N, dtype=torch.float64, device=dev)
    w = torch.tensor(z0, dtype=torch.float64, device=dev)
    Aw = torch.empty_like(w)
    S.apply(w, Aw)
    nrm = S.dot(w, Aw) ** 0.5
    V[0], AV[0] = w / nrm, Aw / nrm
    diag, off = [], []
    for j in range(steps):
        w = V[j].clone()
        S.vcycle(zero, w)                      # w = E_k v_j
        diag.append(S.dot(w, AV[j]))
        for _ in range(2):                     # classical Gram-Schmidt, twice
            w -= V[: j + 1].T @ (AV[: j + 1] @ w)
        S.apply(w, Aw)
        b = max(S.dot(w, Aw), 0.0) ** 0.5
        if j == steps - 1 or b < 1e-14 * abs(diag[0]):
            break
        off.append(b)
        V[j + 1], AV[j + 1] = w / b, Aw / b
    k = len(diag)
    T = np.diag(diag) + np.diag(off[: k - 1], 1) + np.diag(off[: k - 1], -1)
    return float(np.max(np.abs(np.linalg.eigvalsh(T))))


def table_row(k: int, alpha: float, ms=(1, 2, 3, 4, 5), smoother: int = ndmg.SMOOTHER_VERTEX,
              steps: int = 150) -> list[float]:
    """One row of Table 2 (vertex) or Table 1 (edge): level k, all m."""
    n = 2 ** (k + 1)
    return [contraction(n, alpha, m, smoother=smoother, steps=steps) for m in ms]


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--k", type=int, nargs="+", default=[1, 2, 3, 4])
    p.add_argument("--alpha", type=float, nargs="+", default=[0.01, 0.1, 1.0, 10.0, 100.0])
    p.add_argument("--m", type=int, nargs="+", default=[1, 2, 3, 4, 5])
    p.add_argument("--smoother", choices=["vertex", "edge"], default="vertex")
    p.add_argument("--steps", type=int, default=150)
    a = p.parse_args(argv)
    sm = ndmg.SMOOTHER_VERTEX if a.smoother == "vertex" else ndmg.SMOOTHER_EDGE
    print("alpha k " + " ".join(f"m={m}" for m in a.m))
    for al in a.alpha:
        for k in a.k:
            row = table_row(k, al, a.m, sm, a.steps)
            print(f"{al:g} {k} " + " ".join(f"{x:.3f}" for x in row), flush=True)


if __name__ == "__main__":
    main()
