"""Pins for the FP64 CPU oracle: every check compares it with something fixed
by the paper or by mathematics, never with itself (arXiv 2205.05840).

Each group names the passage it pins and the kind of mistake it would catch.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import hcurl, mg
from paper_2205_05840_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def _sine(L=1.0):
    def u(x, y, z):
        s = lambda t: np.sin(np.pi * t / L)
        return np.stack([s(y) * s(z), s(z) * s(x), s(x) * s(y)])
    return u


# ---------------------------------------------------------------- Sec. 2 --

def test_dof_counts_and_numbering():
    # interior edges only (zero tangential trace, eq. (1))
    assert [hcurl.num_edges(n) for n in (2, 4, 8, 32)] == [6, 108, 1176, 92256]
    for n in (2, 3, 5):
        d, i, j, k = hcurl.edge_coords(n)
        idx = hcurl.edge_index(n, d, i, j, k)
        assert (idx == np.arange(hcurl.num_edges(n))).all()
        d2, i2, j2, k2 = hcurl.edge_coords_of(n, idx)
        assert (d2 == d).all() and (i2 == i).all() and (j2 == j).all() and (k2 == k).all()
    # boundary edges are excluded
    assert hcurl.edge_index(4, 0, 0, 0, 1) == -1 and hcurl.edge_index(4, 1, 4, 0, 1) == -1


def test_nodal_basis_is_dual_to_edge_averages():
    # eq. (NDdof): lambda_e(phi_e') = delta_ee'
    h = 0.37
    B = hcurl.nodal_basis(h)
    for e in range(12):
        for f, (d, off) in enumerate(hcurl.LOCAL_EDGES):
            assert abs(hcurl._edge_average(B[:, e], h, d, off) - (e == f)) < 1e-12


def test_element_matrices_closed_form():
    # Closed forms of the lowest-order hexahedral element on a cube of side h,
    # derived by hand from phi = l_a(y) l_b(z) e_x etc. with
    # int l_a l_c = h m_ac, m = [[1/3,1/6],[1/6,1/3]], l_a' = s_a / h, s = (-1, 1).
    h = 0.3
    K, M = hcurl.element_matrices(h)
    m = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    s = np.array([-1.0, 1.0])
    Kc = np.zeros((12, 12))
    Mc = np.zeros((12, 12))
    E = hcurl.LOCAL_EDGES
    for p, (d1, o1) in enumerate(E):
        for q, (d2, o2) in enumerate(E):
            # transverse offsets (cyclic order)
            a, b = o1[(d1 + 1) % 3], o1[(d1 + 2) % 3]
            c, e = o2[(d2 + 1) % 3], o2[(d2 + 2) % 3]
            if d1 == d2:
                Mc[p, q] = h ** 3 * m[a, c] * m[b, e]
                Kc[p, q] = h * (m[a, c] * s[b] * s[e] + s[a] * s[c] * m[b, e])
            elif d2 == (d1 + 1) % 3:
                # edge 1 along x at (y=a, z=b); edge 2 along y at (z=c, x=e):
                # curl1 . curl2 = -(s_a/h) l_b(z) * (s_e/h) l_c(z)
                Kc[p, q] = -h * s[a] * s[e] * m[b, c]
    for p, (d1, _) in enumerate(E):
        for q, (d2, _) in enumerate(E):
            if d2 == (d1 + 2) % 3:
                Kc[p, q] = Kc[q, p]      # symmetry of the curl-curl form
    assert np.allclose(M, Mc, atol=1e-15)
    assert np.allclose(K, Kc, atol=1e-14)


@pytest.mark.parametrize("n,lmin", [(2, 0.0556), (4, 2.90e-3), (8, 2.51e-4)])
def test_operator_spd(n, lmin):
    # eq. (3): a(.,.) is symmetric and coercive for alpha > 0
    A = hcurl.assemble(n, 1.0, 1.0, 1.0)
    assert abs(A - A.T).max() == 0.0
    ev = np.linalg.eigvalsh(A.toarray())
    assert ev[0] > 0
    assert abs(ev[0] - lmin) / lmin < 5e-3
    np.linalg.cholesky(A.toarray())


@pytest.mark.parametrize("n", [3, 4, 6])
def test_de_rham(n):
    # the curl of the edge interpolant of a nodal gradient vanishes
    K, _ = hcurl.assemble_parts(n, 1.0)
    G = hcurl.nodal_gradient(n, 1.0)
    assert abs(K @ G).max() < 1e-13 * abs(K).max() * n


@pytest.mark.parametrize("n", [4, 8])
def test_sine_eigenpairs(n):
    # The sine field is an exact discrete eigenvector of both matrices:
    # M Pi u = h^3 mu^2 Pi u, K Pi u = 8 h sin^2(pi h/2) mu Pi u, mu = (2 + cos pi h)/3.
    h = 1.0 / n
    Pu = hcurl.edge_interpolant(n, 1.0, _sine())
    K, M = hcurl.assemble_parts(n, 1.0)
    mu = (2.0 + np.cos(np.pi * h)) / 3.0
    assert np.allclose(M @ Pu, h ** 3 * mu ** 2 * Pu, atol=1e-15)
    assert np.allclose(K @ Pu, 8 * h * np.sin(np.pi * h / 2) ** 2 * mu * Pu, atol=1e-14)
    assert np.allclose(Pu, inputs.sine_interpolant(n), atol=1e-14)


@pytest.mark.parametrize("n,L,alpha", [(4, 1.0, 1.0), (6, 1.0, 0.01), (4, 2.0, 10.0)])
def test_manufactured_load_matches_quadrature(n, L, alpha):
    # <f_h, phi_e> = (f, phi_e) (Sec. 2): high-order quadrature vs closed form
    u = _sine(L)
    c = 2 * np.pi ** 2 * alpha / L ** 2 + 1.0
    fq = hcurl.load_vector(n, L, lambda x, y, z: c * u(x, y, z), nq=8)
    assert np.allclose(fq, inputs.manufactured_load(n, L, alpha, 1.0), atol=1e-13, rtol=1e-11)


@pytest.mark.parametrize("alpha", [0.01, 1.0, 100.0])
def test_manufactured_discrete_solution_and_convergence(alpha):
    # The discrete solution of the manufactured problem is c Pi u with a closed
    # form c; c - 1 = O(h^2) and the L2 field error is O(h).
    cs, errs = [], []
    for n in (4, 8, 16):
        h = 1.0 / n
        f = inputs.manufactured_load(n, 1.0, alpha, 1.0)
        A = hcurl.assemble(n, 1.0, alpha, 1.0)
        uh = spla.spsolve(A.tocsc(), f)
        Pu = inputs.sine_interpolant(n)
        mu = (2.0 + np.cos(np.pi * h)) / 3.0
        sig = (np.sin(np.pi * h / 2) / (np.pi * h / 2)) ** 2
        c = (2 * np.pi ** 2 * alpha + 1) * sig ** 2 / (8 * alpha * np.sin(np.pi * h / 2) ** 2 * mu / h ** 2 + mu ** 2)
        assert np.allclose(uh, c * Pu, rtol=1e-9, atol=1e-12)
        cs.append(abs(c - 1.0))
        _, M = hcurl.assemble_parts(n, 1.0)
        # ||u - u_h||_L2^2 = ||u||^2 - 2 (u, u_h) + (u_h, u_h); (u, phi_e) = load / (2pi^2 alpha+1)
        uu = 3 * 0.25
        ufl = inputs.manufactured_load(n, 1.0, 0.0, 1.0)
        errs.append(np.sqrt(max(uu - 2 * ufl @ uh + uh @ (M @ uh), 0.0)))
    assert cs[0] / cs[1] > 3.5 and cs[1] / cs[2] > 3.8          # O(h^2)
    assert errs[0] / errs[1] > 1.8 and errs[1] / errs[2] > 1.9  # O(h)


# -------------------------------------------------------------- Sec. 3.1 --

@pytest.mark.parametrize("nc", [2, 3, 4])
def test_galerkin_identity(nc):
    # nested spaces, I_{k-1}^k = natural injection: P^T A_h P = A_H (eq. F2C)
    for alpha, beta in ((1.0, 1.0), (0.01, 2.0)):
        Af = hcurl.assemble(2 * nc, 1.0, alpha, beta)
        Ac = hcurl.assemble(nc, 1.0, alpha, beta)
        P = mg.prolongation(nc, 1.0)
        assert abs(P.T @ Af @ P - Ac).max() < 1e-14 * abs(Ac).max() * 10


def test_prolongation_weights():
    # fine x-edge values of a coarse x basis function: 1 on the two halves of
    # the coarse edge, 1/2 one fine row away, 1/4 diagonally
    P = mg.prolongation(4, 1.0)
    vals = np.unique(np.round(P.data, 14))
    assert set(vals.tolist()) == {0.25, 0.5, 1.0}
    E = hcurl.edge_index(4, 0, 1, 2, 2)
    col = P[:, E].toarray().ravel()
    nz = np.nonzero(col)[0]
    d, i, j, k = hcurl.edge_coords_of(8, nz)
    assert (d == 0).all() and set(i.tolist()) == {2, 3}
    w = {(jj, kk): col[e] for e, jj, kk in zip(nz, j, k)}
    assert np.allclose([w[(4, 4)], w[(3, 4)], w[(5, 5)]], [1.0, 0.5, 0.25], atol=1e-13)
    assert len(nz) == 18


@pytest.mark.parametrize("n", [2, 4, 8])
def test_coarse_direct_solve(n):
    # MG(0, g, z0, m) = A_0^{-1} g: Cholesky vs sparse LU
    A = hcurl.assemble(n, 1.0, 1.0, 1.0)
    g = inputs.random_load(n, 3)
    x1 = sla.cho_solve(sla.cho_factor(A.toarray()), g)
    x2 = spla.splu(A.tocsc()).solve(g)
    assert np.abs(x1 - x2).max() < 1e-11 * np.abs(x2).max()


# -------------------------------------------------------------- Sec. 3.2 --

def test_index_sets():
    b = mg.bubble_sets(8)
    assert b.shape == (64, 6) and len(np.unique(b)) == 64 * 6      # disjoint
    idx, nI = mg.vertex_patches(8)
    assert idx.shape == (27, 108) and nI == 48
    # every fine edge lies in 2 (coarse edge), 4 (coarse face) or 8 (element
    # interior) vertex patches when far from the boundary
    cnt = np.bincount(idx.ravel(), minlength=hcurl.num_edges(8))
    d, i, j, k = hcurl.edge_coords(8)
    far = (np.minimum.reduce([i, j, k]) >= 3) & (np.maximum.reduce([i, j, k]) <= 4)
    tr_odd = np.where(d == 0, (j % 2) + (k % 2), np.where(d == 1, (k % 2) + (i % 2), (i % 2) + (j % 2)))
    expect = np.array([2, 4, 8])[tr_odd]
    assert (cnt[far] == expect[far]).all()
    e3, nIe = mg.edge_patches(8)
    assert nIe == 24 and all(a.shape[1] == 42 for a in e3)


@pytest.mark.parametrize("kind,nI,nd", [("vertex", 48, 108), ("edge", 24, 42)])
def test_schur_patch_is_harmonic_extension(kind, nI, nd):
    # J_D A_D^{-1} J_D^t = A_patch^{-1} - blockdiag(A_II^{-1}, 0): rank = #interface, PSD,
    # and its range is a-orthogonal to the bubble spaces (eq. vertex/edge space)
    n = 8
    A = hcurl.assemble(n, 1.0, 0.3, 1.0)
    idx = mg.vertex_patches(n)[0] if kind == "vertex" else mg.edge_patches(n)[0][0]
    Ap = A[idx[0]][:, idx[0]].toarray()
    D = mg.SchurPatch(Ap, nI).dense()
    ref = np.linalg.inv(Ap)
    ref[:nI, :nI] -= np.linalg.inv(Ap[:nI, :nI])
    assert np.allclose(D, ref, atol=1e-10 * abs(ref).max())
    ev = np.linalg.eigvalsh(0.5 * (D + D.T))
    assert ev.min() > -1e-10 * ev.max()
    assert (ev > 1e-8 * ev.max()).sum() == nd - nI
    assert abs((Ap @ D)[:nI]).max() < 1e-10       # a(v, w_T) = 0 for v in range


@pytest.mark.parametrize("kind,eta_max", [("vertex", 1 / 8), ("edge", 1 / 12)])
def test_smoother_spectral_bound(kind, eta_max):
    # Sec. 3.2: spectral radius of M^{-1} A <= 1 for eta <= 1/8 (vertex), 1/12 (edge);
    # M^{-1} is symmetric positive definite
    n = 8
    A = hcurl.assemble(n, 1.0, 1.0, 1.0)
    S = mg.Smoother(A, n, kind, eta=eta_max)
    Minv = np.stack([S.apply(e) for e in np.eye(A.shape[0])], axis=1)
    assert np.allclose(Minv, Minv.T, atol=1e-12 * abs(Minv).max())
    assert np.linalg.eigvalsh(0.5 * (Minv + Minv.T)).min() > 0
    lam = np.linalg.eigvals(Minv @ A.toarray()).real.max()
    assert lam <= 1.0 + 1e-10


def _centre_gradient(n, cx, cy, cz):
    """Edge DOFs of grad of the fine nodal hat at the centre of coarse element
    (cx, cy, cz): +-1/h on the 6 edges at that node."""
    z = np.zeros(hcurl.num_edges(n))
    h = 1.0 / n
    c = (2 * cx + 1, 2 * cy + 1, 2 * cz + 1)
    for d in range(3):
        lo = list(c)
        lo[d] -= 1
        z[hcurl.edge_index(n, d, *lo)] = 1.0 / h     # edge ending at the node
        z[hcurl.edge_index(n, d, *c)] = -1.0 / h     # edge starting at the node
    return z


@pytest.mark.parametrize("kind,eta", [("vertex", 1 / 9), ("edge", 1 / 13)])
def test_interior_gradient_eigenmode(kind, eta):
    # grad psi_c lies in N_h^T, is a-orthogonal to the coarse space and to every
    # vertex/edge space, so one V-cycle with g = 0 multiplies it by (1-eta)^(2m)
    for n, m in ((4, 1), (8, 2)):
        H = mg.Hierarchy(n, 1.0, 0.7, 1.0, n0=2, kind=kind, m=m)
        z0 = _centre_gradient(n, 1, 0, 1)
        z1 = H.vcycle(np.zeros_like(z0), z0)
        assert np.allclose(z1, (1 - eta) ** (2 * m) * z0, rtol=1e-12, atol=1e-12 * abs(z0).max())


# -------------------------------------------------------------- Sec. 3.3 / 5 --

def _table2():
    rows = {}
    with open(os.path.join(HERE, "golden", "table2_vertex.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[(float(p[0]), int(p[1]))] = [float(x) for x in p[2:]]
    return rows


@pytest.mark.parametrize("alpha", [0.01, 0.1, 1.0, 10.0, 100.0])
def test_table2_k1_reproduced(alpha):
    # Table 2, k = 1 (4^3 cells on (-1,1)^3, T_0 = 2^3): ||E_1||_a to 3 digits
    ref = _table2()[(alpha, 1)]
    for m in range(1, 6):
        H = mg.Hierarchy(4, 2.0, alpha, 1.0, n0=2, kind="vertex", m=m)
        assert round(mg.contraction_dense(H), 3) == pytest.approx(ref[m - 1], abs=1e-9)


def test_table2_k2_approximate():
    # Table 2, k = 2: the exact ||E_2||_a is within 0.03 of the printed numbers
    # (the printed ones sit ~1.5% lower; read as finite-iteration estimates)
    ref = _table2()[(1.0, 2)]
    for m in (1, 2):
        H = mg.Hierarchy(8, 2.0, 1.0, 1.0, n0=2, kind="vertex", m=m)
        rho = mg.contraction_dense(H)
        assert abs(rho - ref[m - 1]) < 0.03
        assert rho >= (8 / 9) ** (2 * m) - 1e-12      # interior eigenmode lower bound


@pytest.mark.parametrize("alpha,k,m", [(0.01, 1, 3), (100.0, 2, 1), (1.0, 2, 2)])
def test_lanczos_contraction_equals_dense(alpha, k, m):
    # the Lanczos estimate used at k >= 3 (where the dense E_k is out of reach)
    # reproduces the exact ||E_k||_a of the dense error operator
    H = mg.Hierarchy(2 ** (k + 1), 2.0, alpha, 1.0, n0=2, kind="vertex", m=m)
    assert abs(mg.contraction_lanczos(H, steps=150) - mg.contraction_dense(H)) < 1e-10


def test_vcycle_error_operator_spsd_and_contractive():
    # Remark 6: E_k is a-symmetric positive semidefinite; Theorem 10: ||E_k||_a < 1
    H = mg.Hierarchy(8, 1.0, 1.0, 1.0, n0=2, m=1)
    A = H.A[-1].toarray()
    E = mg.error_operator(H)
    AE = A @ E
    assert np.allclose(AE, AE.T, atol=1e-10 * abs(AE).max())
    Lc = np.linalg.cholesky(A)
    ev = np.linalg.eigvalsh(Lc.T @ E @ np.linalg.inv(Lc.T) + (Lc.T @ E @ np.linalg.inv(Lc.T)).T) / 2
    assert ev.min() > -1e-10 and ev.max() < 0.85


def test_vcycle_preconditioner_symmetric():
    # B = MG(k, ., 0, m) is symmetric (R_k a-symmetric): x^T B y = y^T B x
    H = mg.Hierarchy(8, 1.0, 0.5, 1.0, n0=2, m=2)
    rng = np.random.default_rng(5)
    x, y = rng.standard_normal((2, H.A[-1].shape[0]))
    z0 = np.zeros_like(x)
    a, b = x @ H.vcycle(y, z0), y @ H.vcycle(x, z0)
    assert abs(a - b) < 1e-12 * abs(a)


@pytest.mark.slow
def test_h_independent_contraction():
    # Theorem 10: the vertex m=1 contraction does not grow with k
    vals = []
    for n in (4, 8, 16):
        H = mg.Hierarchy(n, 2.0, 1.0, 1.0, n0=2, kind="vertex", m=1)
        vals.append(mg.contraction_power(H, iters=40))
    assert all(0.78 <= v <= 0.81 for v in vals), vals


def test_config1_vcycle_iteration_converges():
    # unit cube 8^3, alpha=1, seed-0 load, 3 levels, m=2: standalone V-cycle to 1e-8
    H = mg.Hierarchy(8, 1.0, 1.0, 1.0, n0=2, kind="vertex", m=2)
    f = inputs.random_load(8, 0)
    z, it, hist = mg.vcycle_iteration(H, f, tol=1e-8)
    assert hist[-1] <= 1e-8 and 30 <= it <= 45
    u = spla.spsolve(H.A[-1].tocsc(), f)
    assert np.allclose(z, u, rtol=1e-6, atol=1e-7 * abs(u).max())
    up, itp, rr, _ = mg.pcg(H, f, tol=1e-8)
    assert rr <= 1e-8 and itp < it


def test_adjoint_gradient_matches_finite_differences():
    # dL/dalpha = -lambda^T K u, dL/df = lambda (A symmetric)
    n = 8
    f = inputs.random_load(n, 0)
    ut = 1e-2 * inputs.random_target(n, 1)
    alpha = 0.7

    def loss(a, ff):
        u = mg.solve_direct(n, 1.0, a, 1.0, ff)
        return 0.5 * float((u - ut) @ (u - ut))

    H = mg.Hierarchy(n, 1.0, alpha, 1.0, n0=2, m=2)
    Lv, lam, dalpha, _ = mg.loss_and_grad(H, f, ut)
    eps = 1e-4 * alpha
    fd = (loss(alpha + eps, f) - loss(alpha - eps, f)) / (2 * eps)
    assert abs(dalpha - fd) < 1e-5 * abs(fd)
    v = np.random.default_rng(9).standard_normal(f.size)
    t = 1e-3
    fdf = (loss(alpha, f + t * v) - loss(alpha, f - t * v)) / (2 * t)
    assert abs(lam @ v - fdf) < 1e-5 * abs(fdf)


# ------------------------------------------------- Sec. 2, element by element --

def _boundary_adjacent_rows(n):
    """Every edge with a node or segment on the first or last interior plane
    of some axis (those are the rows whose element sums meet the boundary)."""
    d, i, j, k = hcurl.edge_coords(n)
    near = np.zeros(d.shape, dtype=bool)
    for c in (i, j, k):
        near |= (c <= 1) | (c >= n - 2)
    return np.nonzero(near)[0]


@pytest.mark.parametrize("n", [4, 7, 16])
def test_apply_rows_equals_assembled_rows(n):
    # (A_h u)[rows] summed element by element (used for the expected values of
    # sampled rows on grids too large to assemble) against the sparse assembly
    # of Sec. 2, with alpha, beta != 1 so that a dropped or swapped term shows
    alpha, beta, L = 0.37, 2.9, 1.3
    A = hcurl.assemble(n, L, alpha, beta)
    u = np.random.default_rng(n).standard_normal(hcurl.num_edges(n))
    rng = np.random.default_rng(100 + n)
    rows = np.unique(np.concatenate([_boundary_adjacent_rows(n),
                                     rng.choice(hcurl.num_edges(n), size=min(200, hcurl.num_edges(n)),
                                                replace=False)]))
    got = hcurl.apply_rows(n, L, alpha, beta, u, rows)
    ref = (A @ u)[rows]
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(A).max() * np.abs(u).max() * 33


@pytest.mark.parametrize("n", [32, 64])
def test_apply_rows_sine_eigenpair(n):
    # the closed-form eigenpair of Sec. 2 at sizes the assembly is not used at:
    # A Pi u = (alpha 8 h sin^2(pi h / 2) mu + beta h^3 mu^2) Pi u on the unit cube
    alpha, beta = 3.0, 0.5
    h = 1.0 / n
    mu = (2.0 + np.cos(np.pi * h)) / 3.0
    lam = alpha * 8 * h * np.sin(np.pi * h / 2) ** 2 * mu + beta * h ** 3 * mu ** 2
    Pu = inputs.sine_interpolant(n)
    rows = np.unique(np.concatenate([_boundary_adjacent_rows(n)[::7],
                                     np.random.default_rng(n).choice(Pu.size, 3000, replace=False)]))
    got = hcurl.apply_rows(n, 1.0, alpha, beta, Pu, rows)
    assert np.abs(got - lam * Pu[rows]).max() <= 1e-12 * lam


@pytest.mark.parametrize("n,alpha", [(8, 1.0), (16, 0.05), (16, 50.0)])
def test_pcg_solution_equals_direct_solve(n, alpha):
    # PCG with the V-cycle preconditioner (textbook Hestenes-Stiefel with
    # B = MG(K, ., 0, m)) returns the solution of A u = f: compared with a
    # sparse direct solve and with the true (not recursively updated) residual
    H = mg.Hierarchy(n, 1.0, alpha, 1.0, n0=2, kind="vertex", m=2)
    f = inputs.random_load(n, 3)
    u, it, rr, hist = mg.pcg(H, f, tol=1e-10)
    A = H.A[-1]
    ud = spla.spsolve(A.tocsc(), f)
    true_rel = np.linalg.norm(f - A @ u) / np.linalg.norm(f)
    assert rr <= 1e-10 and true_rel <= 2e-10, (rr, true_rel)
    # the error is bounded by cond(A) times the residual; the sizes here keep
    # cond(A) below 1e3
    assert np.linalg.norm(u - ud) <= 1e-7 * np.linalg.norm(ud)
    # and PCG needs fewer iterations than the standalone V-cycle contraction allows
    assert it < 40
