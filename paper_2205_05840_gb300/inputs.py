"""Seeded synthetic inputs shared by the tests, the smoke check and the
benchmark.  This module holds no solver arithmetic: it only draws random
load vectors and evaluates the closed-form load of one manufactured field.

Load vectors live on the dual side (<f_h, phi_e> per interior edge) in the
canonical edge order of the library (x-edges, then y-edges, then z-edges;
see include/ndmg.h).
"""
from __future__ import annotations

import numpy as np


def num_edges(n: int) -> int:
    return 3 * n * (n - 1) ** 2


def random_load(n: int, seed: int = 0, nrhs: int = 1) -> np.ndarray:
    """i.i.d. uniform[-1, 1] per-edge load; right-hand side r uses seed+r.
    Shape (N,) for nrhs == 1, else (nrhs, N)."""
    N = num_edges(n)
    if nrhs == 1:
        return np.random.default_rng(seed).uniform(-1.0, 1.0, N)
    return np.stack([np.random.default_rng(seed + r).uniform(-1.0, 1.0, N) for r in range(nrhs)])


def random_target(n: int, seed: int = 1) -> np.ndarray:
    """Seeded u_target for the differentiable-solve loss."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, num_edges(n))


def checker_field(n: int, block: int, lo: float = 1.0, hi: float = 100.0) -> np.ndarray:
    """Curl-curl coefficient per hexahedron: two materials in a checkerboard of
    block^3-cell cubes (cell (i, j, k) at (k n + j) n + i)."""
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.where(((i // block) + (j // block) + (k // block)) % 2 == 0, lo, hi).ravel().astype(float)


def inclusion_field(n: int, lo: float = 1.0, hi: float = 100.0) -> np.ndarray:
    """A cube of material hi (cells [n/4, 3n/4)^3) inside material lo."""
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    a, b = n // 4, 3 * n // 4
    inside = (i >= a) & (i < b) & (j >= a) & (j < b) & (k >= a) & (k < b)
    return np.where(inside, hi, lo).ravel().astype(float)


def random_field(n: int, seed: int = 0, lo: float = 0.1, hi: float = 10.0) -> np.ndarray:
    """Log-uniform coefficient in [lo, hi] drawn independently for every hexahedron."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n ** 3))


def _edge_nodes(n: int):
    """Lattice coordinates (d, i, j, k) of every interior edge, canonical order."""
    parts = []
    kk, jj, ii = np.meshgrid(np.arange(1, n), np.arange(1, n), np.arange(0, n), indexing="ij")
    parts.append((0, ii.ravel(), jj.ravel(), kk.ravel()))
    kk, jj, ii = np.meshgrid(np.arange(1, n), np.arange(0, n), np.arange(1, n), indexing="ij")
    parts.append((1, ii.ravel(), jj.ravel(), kk.ravel()))
    kk, jj, ii = np.meshgrid(np.arange(0, n), np.arange(1, n), np.arange(1, n), indexing="ij")
    parts.append((2, ii.ravel(), jj.ravel(), kk.ravel()))
    return parts


def sine_interpolant(n: int, L: float = 1.0) -> np.ndarray:
    """Edge values of u = (sin(pi y/L) sin(pi z/L), sin(pi z/L) sin(pi x/L),
    sin(pi x/L) sin(pi y/L)).  The tangential component is constant along
    every edge, so this is the exact edge average."""
    h = L / n
    out = []
    for d, i, j, k in _edge_nodes(n):
        s = lambda t: np.sin(np.pi * t * h / L)
        if d == 0:
            out.append(s(j) * s(k))
        elif d == 1:
            out.append(s(k) * s(i))
        else:
            out.append(s(i) * s(j))
    return np.concatenate(out)


def manufactured_load(n: int, L: float = 1.0, alpha: float = 1.0, beta: float = 1.0) -> np.ndarray:
    """(f, phi_e) for f = curl(alpha curl u) + beta u = (2 pi^2 alpha / L^2 + beta) u
    with the sine field above, integrated exactly: each hat function
    against sin gives h * sinc^2(pi h / 2L) times the nodal value."""
    h = L / n
    t = np.pi * h / (2.0 * L)
    sig = (np.sin(t) / t) ** 2
    return (2.0 * np.pi ** 2 * alpha / L ** 2 + beta) * h ** 3 * sig ** 2 * sine_interpolant(n, L)
