"""The seeded input recipe (paper_2205_05840_gb300/inputs.py) that the tests,
the smoke check and the benchmark share: its draws, its fields and its edge
order, checked against their definitions and the oracle's numbering."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import hcurl
from paper_2205_05840_gb300 import inputs


@pytest.mark.parametrize("n", [2, 5, 8])
def test_edge_order_is_the_oracles(n):
    d, i, j, k = hcurl.edge_coords(n)
    parts = inputs._edge_nodes(n)
    assert np.array_equal(np.concatenate([np.full(p[1].size, p[0]) for p in parts]), d)
    for c, ref in zip((1, 2, 3), (i, j, k)):
        assert np.array_equal(np.concatenate([p[c] for p in parts]), ref)
    assert np.array_equal(hcurl.edge_index(n, d, i, j, k), np.arange(inputs.num_edges(n)))


def test_random_loads_are_the_stated_draws():
    n, N = 6, inputs.num_edges(6)
    f = inputs.random_load(n, 3)
    assert f.shape == (N,) and np.array_equal(f, np.random.default_rng(3).uniform(-1.0, 1.0, N))
    F = inputs.random_load(n, 10, nrhs=4)
    assert F.shape == (4, N)
    for r in range(4):   # right-hand side r draws from seed + r
        assert np.array_equal(F[r], np.random.default_rng(10 + r).uniform(-1.0, 1.0, N))
    assert np.array_equal(inputs.random_target(n, 1), np.random.default_rng(1).uniform(-1.0, 1.0, N))
    assert np.abs(f).max() <= 1.0


def test_coefficient_fields():
    n = 8
    inc = inputs.inclusion_field(n, 1.0, 10.0).reshape(n, n, n)     # [k][j][i]
    assert (inc[2:6, 2:6, 2:6] == 10.0).all() and inc.sum() == 10.0 * 64 + 1.0 * (512 - 64)
    chk = inputs.checker_field(n, 2, 1.0, 100.0).reshape(n, n, n)
    assert chk[0, 0, 0] == 1.0 and chk[0, 0, 2] == 100.0 and chk[2, 2, 2] == 100.0 and chk[0, 2, 2] == 1.0
    assert (chk == 1.0).sum() == (chk == 100.0).sum() == 256
    rnd = inputs.random_field(n, 3, 0.1, 10.0)
    assert rnd.shape == (n ** 3,) and rnd.min() >= 0.1 and rnd.max() <= 10.0
    assert np.array_equal(rnd, np.exp(np.random.default_rng(3).uniform(np.log(0.1), np.log(10.0), n ** 3)))


@pytest.mark.parametrize("n,L", [(4, 1.0), (7, 1.3)])
def test_sine_interpolant_is_the_edge_average_of_the_field(n, L):
    # the tangential component of the sine field is constant along every edge:
    # compare with the oracle's edge interpolant (edge averages by quadrature)
    def u(x, y, z):
        s = lambda t: np.sin(np.pi * t / L)  # noqa: E731
        return [s(y) * s(z), s(z) * s(x), s(x) * s(y)]
    ref = hcurl.edge_interpolant(n, L, u)
    assert np.abs(inputs.sine_interpolant(n, L) - ref).max() < 1e-13
