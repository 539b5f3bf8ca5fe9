"""Pins of the oracle for a curl-curl coefficient that is constant per
hexahedron (jumping coefficients, concluding remarks): facts that hold
whatever the field and do not restate the assembly."""
import numpy as np
import pytest

from oracle import hcurl, mg


def checker(n, block, lo=1.0, hi=100.0):
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.where(((i // block) + (j // block) + (k // block)) % 2 == 0, lo, hi).ravel()


def test_constant_field_is_the_scalar_operator():
    n = 6
    A = hcurl.assemble_field(n, 1.0, np.full(n ** 3, 2.5), 0.7)
    assert abs(A - hcurl.assemble(n, 1.0, 2.5, 0.7)).max() < 1e-14 * abs(A).max()
    H1 = mg.Hierarchy(8, 1.0, 0.7, 1.0, n0=2, m=1)
    H2 = mg.Hierarchy(8, 1.0, np.full(8 ** 3, 0.7), 1.0, n0=2, m=1)
    f = np.random.default_rng(0).standard_normal(H1.A[-1].shape[0])
    z1, z2 = H1.vcycle(f, np.zeros_like(f)), H2.vcycle(f, np.zeros_like(f))
    assert np.abs(z1 - z2).max() < 1e-12 * np.abs(z1).max()


def test_field_operator_de_rham_and_spd():
    # curl grad = 0 cell by cell, so K_alpha G = 0 for any field; A is SPD
    n = 6
    a = np.random.default_rng(1).uniform(0.01, 100.0, n ** 3)
    A = hcurl.assemble_field(n, 1.0, a, 1.0)
    K = hcurl.assemble_field(n, 1.0, a, 0.0)
    G = hcurl.nodal_gradient(n, 1.0)
    assert abs(K @ G).max() < 1e-12 * abs(K).max()
    Ad = A.toarray()
    assert np.allclose(Ad, Ad.T) and np.linalg.eigvalsh(Ad).min() > 0


def test_field_is_local():
    # changing alpha on one hexahedron changes only the rows / columns of its
    # 12 edges (interior ones), by (delta alpha) K_T
    n = 5
    a = np.random.default_rng(2).uniform(0.5, 2.0, n ** 3)
    A0 = hcurl.assemble_field(n, 1.0, a, 1.0)
    b = a.copy()
    cell = (2 * n + 3) * n + 1                 # (i, j, k) = (1, 3, 2)
    b[cell] += 7.0
    D = (hcurl.assemble_field(n, 1.0, b, 1.0) - A0).toarray()
    KT, _ = hcurl.element_matrices(1.0 / n)
    dofs = hcurl._element_dofs(n)[cell]
    ref = np.zeros_like(D)
    for x in range(12):
        for y in range(12):
            if dofs[x] >= 0 and dofs[y] >= 0:
                ref[dofs[x], dofs[y]] += 7.0 * KT[x, y]
    assert np.abs(D - ref).max() < 1e-12 * np.abs(ref).max()


def test_coarsened_field_is_the_cell_mean():
    a = np.arange(4 ** 3, dtype=float)
    c = mg.coarsen_field(a, 4)
    assert c.shape == (8,) and c[0] == np.mean([0, 1, 4, 5, 16, 17, 20, 21])


@pytest.mark.parametrize("m", [1, 2])
def test_interior_gradient_eigenmode_with_jumps(m):
    # curl grad psi = 0, so a(grad psi, v) = beta (grad psi, v) whatever alpha:
    # the interior-gradient mode keeps its exact factor (1 - eta)^(2m)
    n, eta = 8, 1 / 9
    H = mg.Hierarchy(n, 1.0, checker(n, 2), 1.0, n0=2, m=m)
    z0 = np.zeros(hcurl.num_edges(n))
    c = (3, 1, 5)
    for d in range(3):
        lo = list(c)
        lo[d] -= 1
        z0[hcurl.edge_index(n, d, *lo)] = 1.0
        z0[hcurl.edge_index(n, d, *c)] = -1.0
    z1 = H.vcycle(np.zeros_like(z0), z0)
    # exact up to rounding, which the local solves amplify by their condition
    # number (~ alpha / h^2 = 6400 here)
    assert np.allclose(z1, (1 - eta) ** (2 * m) * z0, rtol=0, atol=1e-10)


def test_jumping_field_error_operator_spsd_and_contractive():
    # the V-cycle error operator stays a-self-adjoint PSD with norm < 1 for a
    # coefficient jumping by 10^4 between 2x2x2 blocks
    H = mg.Hierarchy(8, 1.0, checker(8, 2, 0.01, 100.0), 1.0, n0=2, m=1)
    A = H.A[-1].toarray()
    E = mg.error_operator(H)
    AE = A @ E
    assert np.allclose(AE, AE.T, atol=1e-9 * abs(AE).max())
    rho = mg.contraction_dense(H)
    assert (8 / 9) ** 2 - 1e-9 <= rho < 0.95


def test_cell_gradient_finite_differences():
    # dL/dalpha_T = -lambda^T K_T u against central differences of the loss
    # (direct solves), and the weighted sum identity sum_T alpha_T g_T = -lambda^T K_alpha u
    n = 4
    rng = np.random.default_rng(3)
    a = np.exp(rng.uniform(np.log(0.1), np.log(10.0), n ** 3))
    N = hcurl.num_edges(n)
    f, ut = rng.uniform(-1, 1, N), 0.1 * rng.uniform(-1, 1, N)
    L0, g, u = mg.loss_and_grad_field(n, 1.0, a, 0.8, f, ut)
    for cell in (0, 21, 42, 63):
        eps = 1e-3 * a[cell]                   # O(eps^2) truncation ~1e-7 relative
        ap, am = a.copy(), a.copy()
        ap[cell] += eps
        am[cell] -= eps
        fd = (mg.loss_and_grad_field(n, 1.0, ap, 0.8, f, ut)[0] - mg.loss_and_grad_field(n, 1.0, am, 0.8, f, ut)[0]) / (2 * eps)
        assert abs(fd - g[cell]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), cell
    lam = rng.standard_normal(N)
    K = hcurl.assemble_field(n, 1.0, a, 0.0)
    gc = mg.grad_cells(n, 1.0, lam, u)
    assert abs(a @ gc + lam @ (K @ u)) < 1e-12 * (np.abs(lam) @ np.abs(K @ u))


@pytest.mark.parametrize("kind", ["vertex", "edge"])
def test_grouped_smoother_equals_patchwise_solves(kind):
    # the smoother groups equal local matrices; the same sum of local solves
    # done patch by patch straight from the assembled matrix (the vertex or
    # edge term as A_p^{-1} minus the interior solves of the subdomains inside)
    n = 8
    a = checker(n, 2, 0.5, 20.0)
    A = hcurl.assemble_field(n, 1.0, a, 1.0).tocsr()
    Sm = mg.Smoother(A, n, kind, varying=True)
    r = np.random.default_rng(4).standard_normal(A.shape[0])
    ref = np.zeros_like(r)
    bub = mg.bubble_sets(n)
    for b in bub:
        ref[b] += np.linalg.solve(A[b][:, b].toarray(), r[b])
    lists = [mg.vertex_patches(n)[0]] if kind == "vertex" else list(mg.edge_patches(n)[0])
    for idx in lists:
        for p in idx:
            Ap = A[p][:, p].toarray()
            y = np.linalg.solve(Ap, r[p])
            # remove the interior-space part: subdomains wholly inside the patch
            inside = [b for b in bub if set(b) <= set(p)]
            for b in inside:
                pos = [list(p).index(e) for e in b]
                y[pos] -= np.linalg.solve(A[b][:, b].toarray(), r[b])
            ref[p] += y
    eta = 1.0 / 9.0 if kind == "vertex" else 1.0 / 13.0
    assert np.abs(Sm.apply(r) - eta * ref).max() < 1e-10 * np.abs(eta * ref).max()
