"""FP64 CPU oracle: lowest-order hexahedral Nedelec discretisation.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library.

What it follows (arXiv 2205.05840):
  * eq. (1), (3)-(4): a(w, v) = alpha (curl w, curl v) + beta (w, v), with
    zero tangential trace on the boundary (beta = 1 in the paper; the mass
    coefficient of the implicit Maxwell step, eq. (Maxwell timestep), is kept
    as a parameter).
  * Sec. 2, eq. (nedlec form): on each hexahedron the field is
    (a1 + a2 y + a3 z + a4 yz, b1 + b2 z + b3 x + b4 zx, c1 + c2 x + c3 y + c4 xy).
  * Sec. 2, eq. (NDdof): the degree of freedom of an edge is the average
    tangential component; the nodal basis is dual to those functionals.
  * Sec. 2: A_h u_h = f_h with <A_h w, v> = a(w, v) and <f_h, v> = (f, v).

The element matrices are obtained the long way round on purpose: the 12
monomial coefficients of the ND(T) field are mapped to the 12 edge averages,
that 12x12 map is inverted to get the nodal basis, and mass and curl-curl are
integrated with a 2-point Gauss rule per axis (exact for these polynomials).
No closed form is used here; tests compare the result against closed forms.

Box: [0, L]^3 with n hexahedra per side, h = L / n.  Only interior edges carry
unknowns (zero tangential trace).  Canonical edge order (all edges oriented
along +axis):
  x-edges: segment i in [0, n), nodes j, k in [1, n-1];
           index ((k-1)(n-1) + (j-1)) n + i
  y-edges: node i in [1, n-1], segment j in [0, n), node k in [1, n-1];
           index n(n-1)^2 + ((k-1) n + j)(n-1) + (i-1)
  z-edges: nodes i, j in [1, n-1], segment k in [0, n);
           index 2n(n-1)^2 + (k(n-1) + (j-1))(n-1) + (i-1)
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# --------------------------------------------------------------------------
# DOF numbering
# --------------------------------------------------------------------------


def num_edges(n: int) -> int:
    """Number of interior edges of an n^3 box mesh."""
    return 3 * n * (n - 1) ** 2


def edge_index(n: int, d, i, j, k):
    """Canonical index of the edge of direction d (0=x, 1=y, 2=z) with
    lattice coordinates (i, j, k); -1 where the edge lies on the boundary
    or outside the box.  Works elementwise on integer arrays."""
    d = np.asarray(d)
    i = np.asarray(i)
    j = np.asarray(j)
    k = np.asarray(k)
    n1 = n - 1
    b = n * n1 * n1
    # segment coordinate along the edge direction, node coordinates across it
    seg = np.where(d == 0, i, np.where(d == 1, j, k))
    na = np.where(d == 0, j, np.where(d == 1, k, i))   # first transverse node
    nb = np.where(d == 0, k, np.where(d == 1, i, j))   # second transverse node
    ok = (seg >= 0) & (seg < n) & (na >= 1) & (na <= n1) & (nb >= 1) & (nb <= n1)
    ix = ((k - 1) * n1 + (j - 1)) * n + i
    iy = b + ((k - 1) * n + j) * n1 + (i - 1)
    iz = 2 * b + (k * n1 + (j - 1)) * n1 + (i - 1)
    idx = np.where(d == 0, ix, np.where(d == 1, iy, iz))
    return np.where(ok, idx, -1)


def edge_coords(n: int):
    """(d, i, j, k) arrays for every interior edge, in canonical order."""
    n1 = n - 1
    out = []
    # x-edges: i fastest, then j, then k
    k, j, i = np.meshgrid(np.arange(1, n), np.arange(1, n), np.arange(0, n), indexing="ij")
    out.append((np.zeros(i.size, int), i.ravel(), j.ravel(), k.ravel()))
    k, j, i = np.meshgrid(np.arange(1, n), np.arange(0, n), np.arange(1, n), indexing="ij")
    out.append((np.ones(i.size, int), i.ravel(), j.ravel(), k.ravel()))
    k, j, i = np.meshgrid(np.arange(0, n), np.arange(1, n), np.arange(1, n), indexing="ij")
    out.append((np.full(i.size, 2), i.ravel(), j.ravel(), k.ravel()))
    d = np.concatenate([o[0] for o in out])
    ii = np.concatenate([o[1] for o in out])
    jj = np.concatenate([o[2] for o in out])
    kk = np.concatenate([o[3] for o in out])
    assert d.size == num_edges(n) and n1 >= 0
    return d, ii, jj, kk


# --------------------------------------------------------------------------
# ND(T) element: nodal basis from the monomial form and the edge averages
# --------------------------------------------------------------------------

# Local edges of a cube [0,h]^3, 4 per direction.  Entry = (direction,
# offset of the edge's start vertex in units of h).
LOCAL_EDGES = []
for _d in range(3):
    for _a in range(2):
        for _b in range(2):
            # transverse axes of direction d, in cyclic order (d+1, d+2)
            off = [0, 0, 0]
            off[(_d + 1) % 3] = _a
            off[(_d + 2) % 3] = _b
            LOCAL_EDGES.append((_d, tuple(off)))

_GAUSS2 = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])   # on [0, 1]
_GW2 = np.array([0.5, 0.5])


def _nd_field(coef, x, y, z):
    """Evaluate the ND(T) field with the 12 coefficients of eq. (nedlec form)
    (a1..a4, b1..b4, c1..c4) at points; returns (3, npts)."""
    a, b, c = coef[0:4], coef[4:8], coef[8:12]
    ux = a[0] + a[1] * y + a[2] * z + a[3] * y * z
    uy = b[0] + b[1] * z + b[2] * x + b[3] * z * x
    uz = c[0] + c[1] * x + c[2] * y + c[3] * x * y
    return np.stack([ux, uy, uz])


def _nd_curl(coef, x, y, z):
    """curl of the ND(T) field, from the derivatives of its monomials."""
    a, b, c = coef[0:4], coef[4:8], coef[8:12]
    dy_uz = c[2] + c[3] * x
    dz_uy = b[1] + b[3] * x
    dz_ux = a[2] + a[3] * y
    dx_uz = c[1] + c[3] * y
    dx_uy = b[2] + b[3] * z
    dy_ux = a[1] + a[3] * z
    one = np.ones_like(x)
    return np.stack([(dy_uz - dz_uy) * one, (dz_ux - dx_uz) * one, (dx_uy - dy_ux) * one])


def _edge_average(coef, h, d, off):
    """lambda_e of eq. (NDdof): mean tangential component along the local
    edge (direction d, start vertex off*h), by a 2-point Gauss rule."""
    s = _GAUSS2 * h
    p = [np.full(2, off[0] * h), np.full(2, off[1] * h), np.full(2, off[2] * h)]
    p[d] = p[d] + s
    val = _nd_field(coef, p[0], p[1], p[2])[d]
    return float(np.dot(_GW2, val))


def nodal_basis(h: float) -> np.ndarray:
    """12x12 matrix whose column e holds the monomial coefficients of the
    nodal basis function phi_e on [0,h]^3 (lambda_e'(phi_e) = delta)."""
    V = np.zeros((12, 12))
    for c in range(12):
        coef = np.zeros(12)
        coef[c] = 1.0
        for e, (d, off) in enumerate(LOCAL_EDGES):
            V[e, c] = _edge_average(coef, h, d, off)
    return np.linalg.inv(V)


def element_matrices(h: float):
    """(K_T, M_T): 12x12 curl-curl and mass matrices of one cube of side h,
    integrated with the tensor 2-point Gauss rule."""
    B = nodal_basis(h)
    g = _GAUSS2 * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    W = (np.einsum("i,j,k->ijk", _GW2, _GW2, _GW2) * h ** 3).ravel()
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    vals = np.stack([_nd_field(B[:, e], X, Y, Z) for e in range(12)])    # (12,3,q)
    curls = np.stack([_nd_curl(B[:, e], X, Y, Z) for e in range(12)])
    M = np.einsum("adq,bdq,q->ab", vals, vals, W)
    K = np.einsum("adq,bdq,q->ab", curls, curls, W)
    return K, M


# --------------------------------------------------------------------------
# Global assembly
# --------------------------------------------------------------------------


def _element_dofs(n: int):
    """(n^3, 12) global edge index of each local edge of each element (-1 on
    the boundary), elements ordered ex fastest."""
    ez, ey, ex = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    cols = []
    for d, off in LOCAL_EDGES:
        cols.append(edge_index(n, d, ex + off[0], ey + off[1], ez + off[2]))
    return np.stack(cols, axis=1)


def assemble(n: int, L: float = 1.0, alpha: float = 1.0, beta: float = 1.0):
    """Assembled sparse (CSR) matrix A_h = alpha K + beta M of Sec. 2."""
    K, M = assemble_parts(n, L)
    return (alpha * K + beta * M).tocsr()


def assemble_parts(n: int, L: float = 1.0):
    """(K, M): alpha-free curl-curl and mass matrices, CSR."""
    h = L / n
    KT, MT = element_matrices(h)
    dofs = _element_dofs(n)
    N = num_edges(n)
    r = np.repeat(dofs, 12, axis=1).ravel()
    c = np.tile(dofs, (1, 12)).ravel()
    keep = (r >= 0) & (c >= 0)
    ne = dofs.shape[0]
    kv = np.tile(KT.ravel(), ne)[keep]
    mv = np.tile(MT.ravel(), ne)[keep]
    r, c = r[keep], c[keep]
    K = sp.csr_matrix((kv, (r, c)), shape=(N, N))
    M = sp.csr_matrix((mv, (r, c)), shape=(N, N))
    K.sum_duplicates()
    M.sum_duplicates()
    return K, M


def assemble_field(n: int, L: float, alpha_cells: np.ndarray, beta: float = 1.0):
    """A_h for a curl-curl coefficient that is constant on every hexahedron
    (eq. 1 with alpha piecewise constant; the concluding remarks' jumping
    coefficients): sum_T (alpha_T K_T + beta M_T).  alpha_cells: n^3 values,
    hexahedra ordered x fastest (as the elements of _element_dofs)."""
    h = L / n
    a = np.asarray(alpha_cells, dtype=float).ravel()
    if a.size != n ** 3:
        raise ValueError("alpha_cells needs n^3 values")
    KT, MT = element_matrices(h)
    dofs = _element_dofs(n)
    N = num_edges(n)
    r = np.repeat(dofs, 12, axis=1).ravel()
    c = np.tile(dofs, (1, 12)).ravel()
    keep = (r >= 0) & (c >= 0)
    vals = (a[:, None] * KT.ravel()[None, :] + beta * MT.ravel()[None, :]).ravel()
    A = sp.csr_matrix((vals[keep], (r[keep], c[keep])), shape=(N, N))
    A.sum_duplicates()
    return A


def apply_rows(n: int, L: float, alpha: float, beta: float, u: np.ndarray, rows) -> np.ndarray:
    """(A_h u)[rows] by summing the element contributions of the (up to 4)
    hexahedra around each requested edge; usable at any n because it never
    forms A_h."""
    h = L / n
    KT, MT = element_matrices(h)
    AT = alpha * KT + beta * MT
    d, i, j, k = edge_coords_of(n, np.asarray(rows))
    out = np.zeros(len(rows))
    for le, (ld, off) in enumerate(LOCAL_EDGES):
        # an element whose local edge le is the requested edge
        sel = d == ld
        if not np.any(sel):
            continue
        ex = i[sel] - off[0]
        ey = j[sel] - off[1]
        ez = k[sel] - off[2]
        inside = (ex >= 0) & (ex < n) & (ey >= 0) & (ey < n) & (ez >= 0) & (ez < n)
        acc = np.zeros(sel.sum())
        for le2, (d2, off2) in enumerate(LOCAL_EDGES):
            g = edge_index(n, d2, ex + off2[0], ey + off2[1], ez + off2[2])
            ok = inside & (g >= 0)
            val = np.zeros(sel.sum())
            val[ok] = u[g[ok]]
            acc += AT[le, le2] * val
        out[sel] += np.where(inside, acc, 0.0)
    return out


def edge_coords_of(n: int, idx: np.ndarray):
    """Inverse of edge_index for canonical indices idx."""
    n1 = n - 1
    b = n * n1 * n1
    idx = np.asarray(idx, dtype=np.int64)
    d = np.where(idx < b, 0, np.where(idx < 2 * b, 1, 2))
    loc = idx - d * b
    # x: ((k-1) n1 + (j-1)) n + i
    ix_i = loc % n
    ix_j = (loc // n) % n1 + 1
    ix_k = loc // (n * n1) + 1
    # y: ((k-1) n + j) n1 + (i-1)
    iy_i = loc % n1 + 1
    iy_j = (loc // n1) % n
    iy_k = loc // (n1 * n) + 1
    # z: (k n1 + (j-1)) n1 + (i-1)
    iz_i = loc % n1 + 1
    iz_j = (loc // n1) % n1 + 1
    iz_k = loc // (n1 * n1)
    i = np.where(d == 0, ix_i, np.where(d == 1, iy_i, iz_i))
    j = np.where(d == 0, ix_j, np.where(d == 1, iy_j, iz_j))
    k = np.where(d == 0, ix_k, np.where(d == 1, iy_k, iz_k))
    return d, i, j, k


# --------------------------------------------------------------------------
# Load vectors and interpolation
# --------------------------------------------------------------------------


def load_vector(n: int, L: float, f, nq: int = 6) -> np.ndarray:
    """f_h of Sec. 2: <f_h, phi_e> = (f, phi_e), by an nq-point Gauss rule
    per axis on every element.  f maps (x, y, z) arrays to a (3, npts) array."""
    h = L / n
    B = nodal_basis(h)
    gx, gw = np.polynomial.legendre.leggauss(nq)
    gx = (gx + 1.0) * 0.5 * h
    gw = gw * 0.5 * h
    X, Y, Z = np.meshgrid(gx, gx, gx, indexing="ij")
    W = np.einsum("i,j,k->ijk", gw, gw, gw).ravel()
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    phis = np.stack([_nd_field(B[:, e], X, Y, Z) for e in range(12)])   # (12,3,q)
    dofs = _element_dofs(n)
    ez, ey, ex = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ex, ey, ez = ex.ravel() * h, ey.ravel() * h, ez.ravel() * h
    out = np.zeros(num_edges(n))
    chunk = 4096
    for s in range(0, dofs.shape[0], chunk):
        e = slice(s, s + chunk)
        px = ex[e][:, None] + X[None, :]
        py = ey[e][:, None] + Y[None, :]
        pz = ez[e][:, None] + Z[None, :]
        fv = f(px, py, pz)                                  # (3, ne, q)
        loc = np.einsum("dnq,edq,q->ne", fv, phis, W)       # (ne, 12)
        dd = dofs[e]
        ok = dd >= 0
        np.add.at(out, dd[ok], loc[ok])
    return out


def edge_interpolant(n: int, L: float, u) -> np.ndarray:
    """(Pi u)_e = lambda_e(u): average tangential component of the field u
    along every interior edge (5-point Gauss rule along the edge)."""
    h = L / n
    d, i, j, k = edge_coords(n)
    gx, gw = np.polynomial.legendre.leggauss(5)
    gx = (gx + 1.0) * 0.5
    gw = gw * 0.5
    out = np.zeros(d.size)
    for q in range(gx.size):
        px = (i + np.where(d == 0, gx[q], 0.0)) * h
        py = (j + np.where(d == 1, gx[q], 0.0)) * h
        pz = (k + np.where(d == 2, gx[q], 0.0)) * h
        val = u(px, py, pz)
        out += gw[q] * np.choose(d, val)
    return out


def nodal_gradient(n: int, L: float) -> sp.csr_matrix:
    """G: interior nodal values -> edge DOFs of the gradient of the
    piecewise-trilinear nodal field (edge average of d/dt = difference / h)."""
    h = L / n
    n1 = n - 1
    d, i, j, k = edge_coords(n)

    def node(ii, jj, kk):
        ok = (ii >= 1) & (ii <= n1) & (jj >= 1) & (jj <= n1) & (kk >= 1) & (kk <= n1)
        return np.where(ok, ((kk - 1) * n1 + (jj - 1)) * n1 + (ii - 1), -1)

    start = node(i, j, k)
    end = node(i + (d == 0), j + (d == 1), k + (d == 2))
    rows = np.arange(d.size)
    r = np.concatenate([rows[end >= 0], rows[start >= 0]])
    c = np.concatenate([end[end >= 0], start[start >= 0]])
    v = np.concatenate([np.full((end >= 0).sum(), 1.0 / h), np.full((start >= 0).sum(), -1.0 / h)])
    return sp.csr_matrix((v, (r, c)), shape=(d.size, n1 ** 3))
