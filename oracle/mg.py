"""FP64 CPU oracle: V-cycle multigrid with nonoverlapping DD smoothers.

TEST INFRASTRUCTURE ONLY (see oracle/hcurl.py): only tests, the smoke check
and the CPU-baseline legs of the benchmark may import it; it shares no code
with the CUDA library.

Follows arXiv 2205.05840, Sec. 3:
  * Sec. 3.1: nested meshes T_k (h_k = h_{k-1}/2); prolongation I_{k-1}^k is
    the natural injection N_{k-1} -> N_k, restriction is its transpose
    (eq. F2C).  P is built by evaluating the edge functionals of the fine
    mesh (eq. NDdof) on every coarse basis function.
  * Sec. 3.2: interior spaces N_h^T (eq. SubdomainSpace, ATDef), vertex
    spaces N_h^V (eq. vertex space, AVDef), the vertex-based smoother
    M_V^{-1} = eta_V (sum_T J_T A_T^{-1} J_T^t + sum_V J_V A_V^{-1} J_V^t)
    (eq. Preconditioner P), and the edge spaces / edge-based smoother
    (eq. edge space, AEDef, Preconditioner E).
  * Sec. 3.3, Fig. 1: the symmetric V-cycle MG(k, g, z0, m).
  * Sec. 4, eq. (VCycleRecursion): the V-cycle error operator, used to
    measure contraction numbers as ||E_k||_a.

Readings where the paper is terse:
  * E_h^D ("interior edges that are parts of D") is the set of fine interior
    edges in the relative interior of D.  So a coarse element's bubble set is
    the 6 fine edges strictly inside it, a vertex patch holds the 108 fine
    edges interior to the 4x4x4 block of fine cells around the coarse vertex
    (48 in the 8 element interiors, 48 in the 12 face interiors, 12 on the 6
    coarse edges), and an edge patch the 42 fine edges interior to the 2x4x4
    block of the 4 elements around a coarse edge.
  * A_V^{-1} on N_h^V (discrete harmonic extensions of the interface values)
    is computed as a Schur complement: with I = bubble edges, G = interface
    edges of the patch, S = A_GG - A_GI A_II^{-1} A_IG,
    J_V A_V^{-1} J_V^t r = [-A_II^{-1} A_IG x_G ; x_G], x_G = S^{-1}(r_G - A_GI A_II^{-1} r_I).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import hcurl

# --------------------------------------------------------------------------
# Grid transfer (Sec. 3.1)
# --------------------------------------------------------------------------


def prolongation(nc: int, L: float = 1.0) -> sp.csr_matrix:
    """I_{k-1}^k as a sparse matrix (fine x coarse): entry (e, E) is
    lambda_e(phi_E), the fine-edge average of the coarse basis function."""
    nf = 2 * nc
    H = L / nc
    h = L / nf
    B = hcurl.nodal_basis(H)
    d, i, j, k = hcurl.edge_coords(nf)
    # a coarse element that contains each fine edge (clamped into the box)
    ex = np.minimum(i // 2, nc - 1)
    ey = np.minimum(j // 2, nc - 1)
    ez = np.minimum(k // 2, nc - 1)
    gq, gw = np.polynomial.legendre.leggauss(3)
    gq = (gq + 1.0) * 0.5
    gw = gw * 0.5
    rows, cols, vals = [], [], []
    fine_idx = np.arange(d.size)
    for le, (ld, off) in enumerate(hcurl.LOCAL_EDGES):
        # value of local coarse basis function le on each fine edge
        val = np.zeros(d.size)
        for q in range(gq.size):
            px = (i + np.where(d == 0, gq[q], 0.0)) * h - ex * H
            py = (j + np.where(d == 1, gq[q], 0.0)) * h - ey * H
            pz = (k + np.where(d == 2, gq[q], 0.0)) * h - ez * H
            fld = hcurl._nd_field(B[:, le], px, py, pz)
            val += gw[q] * np.choose(d, fld)
        gidx = hcurl.edge_index(nc, ld, ex + off[0], ey + off[1], ez + off[2])
        ok = (gidx >= 0) & (np.abs(val) > 1e-14)
        rows.append(fine_idx[ok])
        cols.append(gidx[ok])
        vals.append(val[ok])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    P = sp.coo_matrix((v, (r, c)), shape=(hcurl.num_edges(nf), hcurl.num_edges(nc))).tocsr()
    # an entry reached from two coarse elements sharing the fine edge is the
    # same number twice (tangential continuity); keep one copy
    P.sum_duplicates()
    cnt = sp.coo_matrix((np.ones_like(v), (r, c)), shape=P.shape).tocsr()
    cnt.sum_duplicates()
    P.data = P.data / cnt.data
    return P


# --------------------------------------------------------------------------
# Subdomain index sets (Sec. 3.2, E_h^D as relative interiors)
# --------------------------------------------------------------------------


def bubble_sets(n: int, s: int = 2) -> np.ndarray:
    """(nc^3, 3 s (s-1)^2) fine edge indices of the interior space N_h^T of
    every subdomain T (an s x s x s block of fine cells; s = 2: the coarse
    elements of Sec. 3.2, 6 edges each), subdomains ordered x fastest, edges
    of a block ordered (direction, k, j, i)."""
    nc = n // s
    cz, cy, cx = np.meshgrid(np.arange(nc), np.arange(nc), np.arange(nc), indexing="ij")
    lo = s * np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    if s == 2:
        cols = []
        for d in range(3):
            for q in range(2):
                o = [1, 1, 1]
                o[d] = q          # segment index inside the block, nodes at the centre
                cols.append(hcurl.edge_index(n, d, lo[:, 0] + o[0], lo[:, 1] + o[1], lo[:, 2] + o[2]))
        out = np.stack(cols, axis=1)
    else:
        out, _, _ = _block_edges(n, lo, lo + s, s)
    assert (out >= 0).all()
    return out


def _block_edges(n, lo, hi, s=2):
    """Fine interior edges strictly inside the axis-aligned block of fine
    cells [lo, hi) (per-axis arrays of shape (P, 3)); returns (P, m) indices
    ordered (direction, k, j, i) and a boolean 'edge is a bubble edge' mask
    w.r.t. the subdomain grid of spacing s (neither transverse node on a
    subdomain face)."""
    P = lo.shape[0]
    idx, bub, kind = [], [], []
    ext = hi[0] - lo[0]
    for d in range(3):
        rng = []
        for ax in range(3):
            if ax == d:
                rng.append(np.arange(0, ext[ax]))          # segments inside
            else:
                rng.append(np.arange(1, ext[ax]))          # interior nodes
        kk, jj, ii = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
        ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
        gi = lo[:, 0:1] + ii[None, :]
        gj = lo[:, 1:2] + jj[None, :]
        gk = lo[:, 2:3] + kk[None, :]
        idx.append(hcurl.edge_index(n, d, gi, gj, gk))
        tr = [gi, gj, gk]
        a, b = tr[(d + 1) % 3], tr[(d + 2) % 3]
        bub.append((a % s != 0) & (b % s != 0))
        kind.append(((a % s != 0).astype(int) + (b % s != 0).astype(int)))
    return np.concatenate(idx, axis=1), np.concatenate(bub, axis=1), np.concatenate(kind, axis=1)


def vertex_patches(n: int, s: int = 2):
    """For every interior vertex V of the subdomain grid (spacing s, x
    fastest): the fine edges of the vertex patch (the 2s x 2s x 2s block
    around V; 108 edges for s = 2, 1176 for s = 4), reordered as [bubble
    edges (I) ; interface edges (G)].  Returns (idx (P, m), nI) with
    nI = 8 * 3 s (s-1)^2."""
    nc = n // s
    m = 3 * 2 * s * (2 * s - 1) ** 2
    nI = 8 * 3 * s * (s - 1) ** 2
    if nc < 2:
        return np.zeros((0, m), dtype=np.int64), nI
    vz, vy, vx = np.meshgrid(np.arange(1, nc), np.arange(1, nc), np.arange(1, nc), indexing="ij")
    v = np.stack([vx.ravel(), vy.ravel(), vz.ravel()], axis=1)
    lo = s * v - s
    hi = s * v + s
    idx, bub, _ = _block_edges(n, lo, hi, s)
    assert idx.shape[1] == m and (idx >= 0).all()
    order = np.argsort(~bub[0], kind="stable")     # same pattern for every patch
    assert bub[0].sum() == nI
    assert (bub == bub[0]).all()
    return idx[:, order], nI


def edge_patches(n: int):
    """For every interior coarse edge E: the 42 fine edges interior to the
    block of the 4 coarse elements around E, ordered [24 bubble ; 18
    interface].  Returns a list of three (P_d, 42) arrays (one per coarse
    edge direction d) and nI=24."""
    nc = n // 2
    out = []
    for d in range(3):
        rng = []
        for ax in range(3):
            rng.append(np.arange(0, nc) if ax == d else np.arange(1, nc))
        vz, vy, vx = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
        v = np.stack([vx.ravel(), vy.ravel(), vz.ravel()], axis=1)
        lo = 2 * v - 2
        hi = 2 * v + 2
        lo[:, d] = 2 * v[:, d]
        hi[:, d] = 2 * v[:, d] + 2
        if v.shape[0] == 0:
            out.append(np.zeros((0, 42), dtype=np.int64))
            continue
        idx, bub, _ = _block_edges(n, lo, hi)
        assert idx.shape[1] == 42 and (idx >= 0).all()
        order = np.argsort(~bub[0], kind="stable")
        assert bub[0].sum() == 24 and (bub == bub[0]).all()
        out.append(idx[:, order])
    return out, 24


# --------------------------------------------------------------------------
# Local solves
# --------------------------------------------------------------------------


def coarsen_field(alpha_cells: np.ndarray, n: int) -> np.ndarray:
    """Curl-curl coefficient of the (n/2)^3 coarse hexahedra: the mean of the
    8 fine ones each contains (reading for coefficients that vary per
    hexahedron; the paper's analysis assumes a constant one)."""
    a = np.asarray(alpha_cells, dtype=float).reshape(n, n, n)      # [k, j, i]
    return a.reshape(n // 2, 2, n // 2, 2, n // 2, 2).mean(axis=(1, 3, 5)).ravel()


def _block_groups(A, idx):
    """Group the subdomains / patches of idx by their local matrix (equal up
    to rounding): returns a list of (patch numbers, local matrix)."""
    groups = {}
    for p in range(idx.shape[0]):
        Ap = A[idx[p]][:, idx[p]].toarray()
        key = np.round(Ap / abs(Ap).max(), 11).tobytes() + np.float64(abs(Ap).max()).round(11).tobytes()
        if key in groups:
            groups[key][0].append(p)
        else:
            groups[key] = ([p], Ap)
    return [(np.array(ps), Ap) for ps, Ap in groups.values()]


def _identical_blocks(A, idx, sample=64, seed=0):
    """Extract A[idx_p, idx_p] for a sample of patches, check they are all
    equal (constant alpha on a uniform grid), return the first one."""
    rng = np.random.default_rng(seed)
    P = idx.shape[0]
    picks = np.unique(np.concatenate([[0, P - 1], rng.integers(0, P, size=min(sample, P))]))
    A0 = A[idx[0]][:, idx[0]].toarray()
    for p in picks:
        Ap = A[idx[p]][:, idx[p]].toarray()
        if not np.allclose(Ap, A0, rtol=1e-13, atol=1e-13 * np.abs(A0).max()):
            raise AssertionError("local matrices differ between subdomains")
    return A0


class SchurPatch:
    """J A_D^{-1} J^t for a discrete-harmonic interface space, as the Schur
    complement of the patch matrix on its bubble block (reading stated in
    the module docstring)."""

    def __init__(self, Ap: np.ndarray, nI: int):
        self.nI = nI
        AII = Ap[:nI, :nI]
        self.AIG = Ap[:nI, nI:]
        self.AGI = Ap[nI:, :nI]
        AGG = Ap[nI:, nI:]
        self.cII = sla.cho_factor(AII)
        S = AGG - self.AGI @ sla.cho_solve(self.cII, self.AIG)
        self.cS = sla.cho_factor(S)

    def apply(self, R: np.ndarray) -> np.ndarray:
        """R: (m, P) restricted residuals (columns = patches)."""
        nI = self.nI
        rI, rG = R[:nI], R[nI:]
        gG = rG - self.AGI @ sla.cho_solve(self.cII, rI)
        xG = sla.cho_solve(self.cS, gG)
        xI = -sla.cho_solve(self.cII, self.AIG @ xG)
        return np.vstack([xI, xG])

    def dense(self) -> np.ndarray:
        return self.apply(np.eye(self.AIG.shape[0] + self.AIG.shape[1]))


class Smoother:
    """M_{V,h}^{-1} (eq. Preconditioner P) or M_{E,h}^{-1} (eq.
    Preconditioner E) on one level."""

    def __init__(self, A: sp.csr_matrix, n: int, kind: str = "vertex", eta: float | None = None, s: int = 2,
                 varying: bool = False):
        """varying: the local matrices differ between subdomains (a
        coefficient that varies per hexahedron); they are then grouped by
        equality and factored once per group."""
        self.kind = kind
        self.eta = eta if eta is not None else (1.0 / 9.0 if kind == "vertex" else 1.0 / 13.0)
        self.N = A.shape[0]
        if n % s:
            raise ValueError(f"level n={n} is not a multiple of the subdomain size s={s}")
        if s != 2 and kind != "vertex":
            raise ValueError("subdomain size s != 2 is built for the vertex-based smoother")
        self.bub = bubble_sets(n, s)
        self.varying = varying
        if varying:
            self.bub_groups = [(ps, sla.cho_factor(AT)) for ps, AT in _block_groups(A, self.bub)]
        else:
            AT = _identical_blocks(A, self.bub)
            self.cT = sla.cho_factor(AT)
        self.patches = []
        if kind == "vertex":
            idx, nI = vertex_patches(n, s)
            if idx.shape[0] and varying:
                for ps, Ap in _block_groups(A, idx):
                    self.patches.append((idx[ps], SchurPatch(Ap, nI)))
            elif idx.shape[0]:
                Ap = _identical_blocks(A, idx)
                self.patches.append((idx, SchurPatch(Ap, nI)))
        elif kind == "edge":
            lists, nI = edge_patches(n)
            for idx in lists:
                if idx.shape[0] and varying:
                    for ps, Ap in _block_groups(A, idx):
                        self.patches.append((idx[ps], SchurPatch(Ap, nI)))
                elif idx.shape[0]:
                    Ap = _identical_blocks(A, idx)
                    self.patches.append((idx, SchurPatch(Ap, nI)))
        else:
            raise ValueError(kind)

    def apply(self, r: np.ndarray) -> np.ndarray:
        """M^{-1} r: every local solve reads the same r; results are summed."""
        out = np.zeros_like(r)
        # sum_T J_T A_T^{-1} J_T^t r ; bubble sets are disjoint
        if self.varying:
            for ps, cT in self.bub_groups:
                b = self.bub[ps]
                out[b.T.ravel()] += sla.cho_solve(cT, r[b].T).ravel()
        else:
            yT = sla.cho_solve(self.cT, r[self.bub].T)      # (edges per block, nT)
            out[self.bub.T.ravel()] += yT.ravel()
        # sum_V J_V A_V^{-1} J_V^t r (or the edge spaces)
        for idx, sp_ in self.patches:
            y = sp_.apply(r[idx].T)                          # (m, P)
            np.add.at(out, idx.T.ravel(), y.ravel())
        return self.eta * out


# --------------------------------------------------------------------------
# Level hierarchy and the V-cycle (Fig. 1)
# --------------------------------------------------------------------------


class Hierarchy:
    """Levels n_0 < n_1 < ... < n_K = n with n_k = 2 n_{k-1}."""

    def __init__(self, n: int, L: float = 1.0, alpha: float = 1.0, beta: float = 1.0,
                 n0: int = 2, kind: str = "vertex", eta: float | None = None, m: int = 2, s: int = 2):
        ns = [n]
        while ns[-1] > n0:
            if ns[-1] % 2:
                raise ValueError("every non-coarsest level needs an even n")
            ns.append(ns[-1] // 2)
        if ns[-1] != n0:
            raise ValueError(f"n={n} does not coarsen to n0={n0}")
        self.ns = ns[::-1]
        self.L, self.alpha, self.beta, self.m = L, alpha, beta, m
        field = np.ndim(alpha) > 0
        if field:
            # a coefficient per finest hexahedron, averaged onto coarser grids
            fields = [np.asarray(alpha, dtype=float).ravel()]
            for nk in ns[:-1]:
                fields.append(coarsen_field(fields[-1], nk))
            self.fields = fields[::-1]
            self.A = [hcurl.assemble_field(nk, L, a, beta) for nk, a in zip(self.ns, self.fields)]
        else:
            self.A = [assemble_cached(nk, L, alpha, beta) for nk in self.ns]
        self.P = [None] + [prolongation(self.ns[k - 1], L) for k in range(1, len(self.ns))]
        self.S = [None] + [Smoother(self.A[k], self.ns[k], kind, eta, s, varying=field)
                           for k in range(1, len(self.ns))]
        self.c0 = sla.cho_factor(self.A[0].toarray())

    @property
    def K(self):
        return len(self.ns) - 1

    def mg(self, k: int, g: np.ndarray, z0: np.ndarray, m: int | None = None) -> np.ndarray:
        """MG(k, g, z0, m) exactly as Fig. 1."""
        m = self.m if m is None else m
        if k == 0:
            return sla.cho_solve(self.c0, g)
        A, S, P = self.A[k], self.S[k], self.P[k]
        z = z0.copy()
        for _ in range(m):
            z = z + S.apply(g - A @ z)
        gbar = P.T @ (g - A @ z)
        z = z + P @ self.mg(k - 1, gbar, np.zeros(P.shape[1]), m)
        for _ in range(m):
            z = z + S.apply(g - A @ z)
        return z

    def vcycle(self, g, z0):
        return self.mg(self.K, g, z0)


_ASM_CACHE: dict = {}


def assemble_cached(n, L, alpha, beta):
    key = (n, L)
    if key not in _ASM_CACHE:
        _ASM_CACHE[key] = hcurl.assemble_parts(n, L)
    K, M = _ASM_CACHE[key]
    return (alpha * K + beta * M).tocsr()


# --------------------------------------------------------------------------
# Solvers built on the V-cycle
# --------------------------------------------------------------------------


def vcycle_iteration(H: Hierarchy, f, tol=1e-8, maxit=500, z0=None):
    """Standalone iteration z_{j+1} = MG(K, f, z_j, m); stops when
    ||f - A z||_2 / ||f||_2 <= tol.  Returns (z, iterations, history)."""
    A = H.A[-1]
    z = np.zeros_like(f) if z0 is None else z0.copy()
    nf = np.linalg.norm(f)
    hist = [np.linalg.norm(f - A @ z) / nf]
    it = 0
    while hist[-1] > tol and it < maxit:
        z = H.vcycle(f, z)
        it += 1
        hist.append(np.linalg.norm(f - A @ z) / nf)
    return z, it, hist


def pcg(H: Hierarchy, f, u0=None, tol=1e-8, maxit=200):
    """Preconditioned CG, B = MG(K, ., 0, m).  Returns (u, iters, relres,
    history)."""
    A = H.A[-1]
    u = np.zeros_like(f) if u0 is None else u0.copy()
    r = f - A @ u
    nf = np.linalg.norm(f)
    hist = [np.linalg.norm(r) / nf]
    if hist[-1] <= tol:
        return u, 0, hist[-1], hist
    z = H.vcycle(r, np.zeros_like(r))
    p = z.copy()
    rz = r @ z
    it = 0
    for it in range(1, maxit + 1):
        q = A @ p
        a = rz / (p @ q)
        u = u + a * p
        r = r - a * q
        hist.append(np.linalg.norm(r) / nf)
        if hist[-1] <= tol:
            break
        z = H.vcycle(r, np.zeros_like(r))
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return u, it, hist[-1], hist


# --------------------------------------------------------------------------
# Contraction numbers (Sec. 5) as ||E_k||_a (eq. VCycleRecursion)
# --------------------------------------------------------------------------


def error_operator(H: Hierarchy, m: int | None = None) -> np.ndarray:
    """Dense E_K: column j is MG(K, 0, e_j, m) (the error after one V-cycle
    started from error e_j)."""
    N = H.A[-1].shape[0]
    zero = np.zeros(N)
    E = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        E[:, j] = H.mg(H.K, zero, e, m)
    return E


def contraction_dense(H: Hierarchy, m: int | None = None) -> float:
    """||E_K||_a: E_K is a-self-adjoint, so its a-norm is the largest
    |eigenvalue| of A^{1/2} E A^{-1/2}."""
    A = H.A[-1].toarray()
    E = error_operator(H, m)
    Lc = np.linalg.cholesky(A)
    Sym = Lc.T @ E @ np.linalg.inv(Lc.T)
    Sym = 0.5 * (Sym + Sym.T)
    return float(np.max(np.abs(np.linalg.eigvalsh(Sym))))


def contraction_power(H: Hierarchy, m: int | None = None, iters=60, seed=0) -> float:
    """||E_K||_a by power iteration in the a-inner product."""
    A = H.A[-1]
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(A.shape[0])
    z /= np.sqrt(z @ (A @ z))
    zero = np.zeros_like(z)
    lam = 0.0
    for _ in range(iters):
        w = H.mg(H.K, zero, z, m)
        lam = float(z @ (A @ w))        # Rayleigh quotient, ||z||_a = 1
        z = w / np.sqrt(w @ (A @ w))
    return lam


def contraction_lanczos(H: Hierarchy, m: int | None = None, steps=40, z0=None, seed=0) -> float:
    """||E_K||_a by the Lanczos process in the a-inner product.

    E_K is a-self-adjoint and a-positive semidefinite (Remark 6), so the
    Krylov space of E_K from z0, orthonormalised in (x, y)_a = x^T A y, gives
    a tridiagonal T whose largest eigenvalue approaches ||E_K||_a from below
    (much faster than the power iteration when the top eigenvalues cluster).
    Every new basis vector is orthogonalised against all previous ones."""
    A = H.A[-1]
    if z0 is None:
        z0 = np.random.default_rng(seed).standard_normal(A.shape[0])
    zero = np.zeros(A.shape[0])
    V, AV = [], []
    diag, off = [], []
    Az = A @ z0
    nrm = np.sqrt(z0 @ Az)
    v, Av = z0 / nrm, Az / nrm
    for j in range(steps):
        V.append(v)
        AV.append(Av)
        w = H.mg(H.K, zero, v, m)                  # w = E_K v
        diag.append(float(w @ Av))
        for vi, Avi in zip(V, AV):                  # (w, v_i)_a = w^T (A v_i)
            w = w - (w @ Avi) * vi
        for vi, Avi in zip(V, AV):                  # second pass: orthogonality to rounding
            w = w - (w @ Avi) * vi
        Aw = A @ w
        b = np.sqrt(max(float(w @ Aw), 0.0))
        if j == steps - 1 or b < 1e-14 * abs(diag[0]):
            break
        off.append(b)
        v, Av = w / b, Aw / b
    T = np.diag(diag) + np.diag(off[:len(diag) - 1], 1) + np.diag(off[:len(diag) - 1], -1)
    return float(np.max(np.abs(np.linalg.eigvalsh(T))))


# --------------------------------------------------------------------------
# Adjoint gradient of L = 0.5 ||u(f, alpha) - u_t||^2
# --------------------------------------------------------------------------


def solve_direct(n, L, alpha, beta, f):
    import scipy.sparse.linalg as spla
    A = assemble_cached(n, L, alpha, beta)
    return spla.spsolve(A.tocsc(), f)


def loss_and_grad(H: Hierarchy, f, u_t, tol=1e-12):
    """L, dL/df = lambda, dL/dalpha = -lambda^T K u with A lambda = u - u_t
    (A symmetric)."""
    u, *_ = pcg(H, f, tol=tol, maxit=500)
    res = u - u_t
    lam, *_ = pcg(H, res, tol=tol, maxit=500)
    K, _ = _ASM_CACHE[(H.ns[-1], H.L)]
    return 0.5 * float(res @ res), lam, -float(lam @ (K @ u)), u


def grad_cells(n: int, L: float, lam, u):
    """-lambda_T^t K_T u_T for every hexahedron T (x fastest): the derivative
    of a(u, lambda) = sum_T alpha_T (curl u, curl lambda)_T + beta (u, lambda)
    in the coefficient of T, from the element matrix of T and the element's
    edge values (zero on boundary edges)."""
    KT, _ = hcurl.element_matrices(L / n)
    dofs = hcurl._element_dofs(n)
    ln = np.where(dofs >= 0, np.asarray(lam)[np.maximum(dofs, 0)], 0.0)
    un = np.where(dofs >= 0, np.asarray(u)[np.maximum(dofs, 0)], 0.0)
    return -np.einsum("ca,ab,cb->c", ln, KT, un)


def loss_and_grad_field(n: int, L: float, alpha_cells, beta, f, u_t):
    """L = 0.5 ||u - u_t||^2 with A(alpha) u = f for a coefficient per
    hexahedron, by sparse direct solves: returns (L, dL/dalpha per cell, u);
    dL/dalpha_T = -lambda^T K_T u with A lambda = u - u_t (A symmetric)."""
    A = hcurl.assemble_field(n, L, alpha_cells, beta).tocsc()
    lu = spla.splu(A)
    u = lu.solve(np.asarray(f, dtype=float))
    res = u - u_t
    lam = lu.solve(res)
    return 0.5 * float(res @ res), grad_cells(n, L, lam, u), u
