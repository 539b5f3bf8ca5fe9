"""Pins of the subdomain-size-4 reading of the vertex-based smoother (the
subdomains are 4 x 4 x 4 blocks of fine cells, the vertex patches the 8 x 8 x 8
blocks around the vertices of that block grid; everything else as in Sec.
3.2).  Each pin is a fact of the construction that a wrong index set,
Schur complement or scaling breaks."""
import numpy as np
import pytest

from oracle import hcurl, mg


def test_index_sets_s4():
    b = mg.bubble_sets(16, 4)
    assert b.shape == (64, 108) and len(np.unique(b)) == 64 * 108        # disjoint
    idx, nI = mg.vertex_patches(16, 4)
    assert idx.shape == (27, 1176) and nI == 864 and 1176 - nI == 312
    # away from the boundary every fine edge lies in 2 (on a block edge),
    # 4 (on a block face) or 8 (inside a block) vertex patches
    cnt = np.bincount(idx.ravel(), minlength=hcurl.num_edges(16))
    d, i, j, k = hcurl.edge_coords(16)
    far = (np.minimum.reduce([i, j, k]) >= 4) & (np.maximum.reduce([i, j, k]) <= 11)
    a_off = np.where(d == 0, j, np.where(d == 1, k, i)) % 4 != 0
    b_off = np.where(d == 0, k, np.where(d == 1, i, j)) % 4 != 0
    expect = np.array([2, 4, 8])[a_off.astype(int) + b_off.astype(int)]
    assert far.sum() > 0 and (cnt[far] == expect[far]).all()
    # the first nI edges of every patch are bubble edges of its 8 blocks
    bub = set(b.ravel().tolist())
    assert all(e in bub for e in idx[:, :nI].ravel()) and not any(e in bub for e in idx[:, nI:].ravel())


def test_schur_patch_s4_is_harmonic_extension():
    n = 8
    A = hcurl.assemble(n, 1.0, 0.3, 1.0)
    idx, nI = mg.vertex_patches(n, 4)
    Ap = A[idx[0]][:, idx[0]].toarray()
    D = mg.SchurPatch(Ap, nI).dense()
    ref = np.linalg.inv(Ap)
    ref[:nI, :nI] -= np.linalg.inv(Ap[:nI, :nI])
    assert np.allclose(D, ref, atol=1e-9 * abs(ref).max())
    ev = np.linalg.eigvalsh(0.5 * (D + D.T))
    assert ev.min() > -1e-10 * ev.max()
    assert (ev > 1e-8 * ev.max()).sum() == 312
    assert abs((Ap @ D)[:nI]).max() < 1e-9 * abs(Ap).max() * abs(D).max()


def test_smoother_s4_spectral_bound():
    # eight colours of vertex patches, as for s = 2: eta <= 1/8 keeps
    # rho(M^{-1} A) <= 1; M^{-1} symmetric positive definite
    n = 8
    A = hcurl.assemble(n, 1.0, 1.0, 1.0)
    S = mg.Smoother(A, n, "vertex", eta=1 / 8, s=4)
    Minv = np.stack([S.apply(e) for e in np.eye(A.shape[0])], axis=1)
    assert np.allclose(Minv, Minv.T, atol=1e-12 * abs(Minv).max())
    assert np.linalg.eigvalsh(0.5 * (Minv + Minv.T)).min() > 0
    lam = np.linalg.eigvals(Minv @ A.toarray()).real.max()
    assert lam <= 1.0 + 1e-10


@pytest.mark.parametrize("m", [1, 2])
def test_interior_gradient_eigenmode_s4(m):
    # grad of the fine nodal hat at a node with odd coordinates strictly inside
    # a 4-block lies in that block's interior space and is a-orthogonal to the
    # coarse space and to every vertex space: one V-cycle with g = 0 scales it
    # by (1 - eta)^(2m)
    n, eta = 8, 1 / 9
    H = mg.Hierarchy(n, 1.0, 0.7, 1.0, n0=4, kind="vertex", m=m, s=4)
    z0 = np.zeros(hcurl.num_edges(n))
    c = (1, 3, 1)
    for dd in range(3):
        lo = list(c)
        lo[dd] -= 1
        z0[hcurl.edge_index(n, dd, *lo)] = 1.0
        z0[hcurl.edge_index(n, dd, *c)] = -1.0
    z1 = H.vcycle(np.zeros_like(z0), z0)
    assert np.allclose(z1, (1 - eta) ** (2 * m) * z0, rtol=1e-12, atol=1e-12)


def test_vcycle_s4_error_operator_spsd_and_contractive():
    # Remark 6 / Theorem 10 carried over: E_k a-symmetric PSD, ||E_k||_a < 1,
    # and no smaller than the interior-gradient factor (1 - eta)^(2m)
    H = mg.Hierarchy(8, 1.0, 1.0, 1.0, n0=4, kind="vertex", m=1, s=4)
    A = H.A[-1].toarray()
    E = mg.error_operator(H)
    AE = A @ E
    assert np.allclose(AE, AE.T, atol=1e-10 * abs(AE).max())
    rho = mg.contraction_dense(H)
    assert (8 / 9) ** 2 - 1e-10 <= rho < 0.9
    assert abs(mg.contraction_lanczos(H, steps=150) - rho) < 1e-10
