"""The mirror-symmetry tables of the patch solves (build_patch_sym in
paper_2205_05840_gb300/csrc/patch_sym.cu), built by a host program and checked
on the CPU.

The FP64 smoother kernel (k_patch_sym) and the FP32 smoother of the small
levels (k_smooth_sym32) apply a patch operator D (eqs. (Preconditioner P) and
(Preconditioner E): J A^{-1} J^t of a vertex, edge or s = 4 subdomain space) as
D = T^t M T: T holds signed sums over the orbits of the patch's edges under the
three reflections through the box centre (entries +-1, one row per orbit and
compatible character), M is block diagonal (one block per character).  The
test decodes the tables the library uploads (the word layout its source
documents), rebuilds T^t M T in FP64 from the stored float pairs of M, and
compares it with the set-up's dense operator; it also checks what the
construction promises: T T^t is diagonal with the orbit sizes, every edge
lies in at most 8 rows, and the vertex patch's blocks have 24, 16, 16, 16, 10,
10, 10 and 6 rows.  The operators come from the set-up (checked against the
oracle in test_setup_host.py).  No kernel is launched, so no GPU is needed."""
from __future__ import annotations

import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2205_05840_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>
#include "kernels.cuh"
using namespace ndmg;
static void wr(const std::string& p, const void* v, size_t bytes) {
  FILE* f = fopen(p.c_str(), "wb"); fwrite(v, 1, bytes, f); fclose(f);
}
static void sym(const std::string& p, const PatchFamily& fam, const std::vector<double>& D) {
  std::vector<uint32_t> blob;
  double dropped = -1.0;
  const bool ok = build_patch_sym(fam, D.data(), &blob, &dropped);
  wr(p + "_D.bin", D.data(), D.size() * sizeof(double));
  wr(p + "_blob.bin", blob.data(), blob.size() * sizeof(uint32_t));
  printf("%s %d %.17g %zu\n", p.c_str(), ok ? 1 : 0, dropped, blob.size());
}
int main(int argc, char** argv) {
  const std::string dir = argv[1];
  const int n = atoi(argv[2]);
  const double L = atof(argv[3]), alpha = atof(argv[4]), beta = atof(argv[5]);
  LocalOps ops;
  build_local_ops(n, L, alpha, beta, &ops, 2);
  sym(dir + "/vertex", vertex_family(n), ops.Dv);
  for (int d = 0; d < 3; ++d) sym(dir + "/edge" + std::to_string(d), edge_family(n, d), ops.De[d]);
  LocalOps ops4;
  build_local_ops(2 * n, L, alpha, beta, &ops4, 4);
  sym(dir + "/sub4", subdomain4_family(2 * n), ops4.AinvT);
  return 0;
}
"""

SOURCES = ["setup.cpp", "kernels.cu", "patch_sym.cu"]
K_HDR = 3 + 3 * 8


@pytest.fixture(scope="module")
def driver(host_build, tmp_path_factory):
    return host_build(DRIVER, SOURCES), str(tmp_path_factory.mktemp("patch_sym_host"))


def _decode(blob: np.ndarray):
    """T (nl x nl, entries -1/0/+1), M (block diagonal, FP64 from its float
    pairs), the block sizes, and the per-edge row lists."""
    nl, nb, mtot = int(blob[0]), int(blob[1]), int(blob[2])
    first = [int(blob[3 + 3 * q]) for q in range(nb)]
    size = [int(blob[4 + 3 * q]) for q in range(nb)]
    moff = [int(blob[5 + 3 * q]) for q in range(nb)]
    T = np.zeros((nl, nl))
    rows_at, edges_at, m_at = K_HDR, K_HDR + 3 * nl, K_HDR + 6 * nl
    row_block = np.zeros(nl, dtype=int)
    for r in range(nl):
        w = blob[rows_at + 3 * r: rows_at + 3 * r + 3]
        mem = np.frombuffer(w[:2].astype("<u4").tobytes(), dtype=np.uint8)
        cnt, signs, blk = int(w[2]) & 0xFF, (int(w[2]) >> 8) & 0xFF, int(w[2]) >> 16
        row_block[r] = blk
        for q in range(cnt):
            T[r, mem[q]] = -1.0 if (signs >> q) & 1 else 1.0
    edge_rows = []
    for e in range(nl):
        w = blob[edges_at + 3 * e: edges_at + 3 * e + 3]
        rr = np.frombuffer(w[:2].astype("<u4").tobytes(), dtype=np.uint8)
        cnt, signs = int(w[2]) & 0xFF, (int(w[2]) >> 8) & 0xFF
        edge_rows.append([(int(rr[q]), -1.0 if (signs >> q) & 1 else 1.0) for q in range(cnt)])
    mf = blob[m_at:m_at + 2 * mtot].astype("<u4").view(np.float32).astype(np.float64)
    mh, ml = mf[:mtot], mf[mtot:]
    M = np.zeros((nl, nl))
    for q in range(nb):
        for r in range(size[q]):
            for s in range(size[q]):
                o = moff[q] + s * size[q] + r
                M[first[q] + r, first[q] + s] = mh[o] + ml[o]
    return T, M, size, row_block, first, edge_rows


@pytest.mark.parametrize("n,L,alpha,beta", [(8, 1.0, 1.0, 1.0), (16, 1.3, 0.37, 2.9), (8, 1.0, 100.0, 1.0)])
def test_symmetry_tables_rebuild_the_patch_operators(driver, n, L, alpha, beta):
    exe, d = driver
    out = os.path.join(d, f"run_{n}_{alpha}")
    os.makedirs(out, exist_ok=True)
    res = subprocess.run([exe, out, str(n), repr(L), repr(alpha), repr(beta)], check=True, capture_output=True,
                         text=True)
    info = {ln.split()[0].rsplit("/", 1)[1]: ln.split()[1:] for ln in res.stdout.splitlines()}
    # (the s = 4 subdomain interior is a 4^3-cell box like the vertex patch;
    # an edge patch, 2 x 4 x 4 cells, has 42 edges)
    expect_blocks = {"vertex": [24, 16, 16, 16, 10, 10, 10, 6], "sub4": [24, 16, 16, 16, 10, 10, 10, 6],
                     "edge0": [12, 8, 8, 5, 4, 2, 2, 1], "edge1": [12, 8, 8, 5, 4, 2, 2, 1],
                     "edge2": [12, 8, 8, 5, 4, 2, 2, 1]}
    for name, (ok, dropped, words) in info.items():
        assert ok == "1", name
        blob = np.fromfile(os.path.join(out, name + "_blob.bin"), dtype=np.uint32)
        assert blob.size == int(words)
        D = np.fromfile(os.path.join(out, name + "_D.bin"), dtype=np.float64)
        nl = int(round(np.sqrt(D.size)))
        D = D.reshape(nl, nl)
        T, M, size, row_block, first, edge_rows = _decode(blob)
        assert int(blob[0]) == nl and sum(size) == nl
        if name in expect_blocks:
            assert sorted(size, reverse=True) == expect_blocks[name]
            if nl == 108:
                assert sum(s * s for s in size) == 1680
        # T: +-1 entries, orthogonal rows, T T^t = the orbit sizes
        assert set(np.unique(T)) <= {-1.0, 0.0, 1.0}
        G = T @ T.T
        assert np.array_equal(G, np.diag(np.diag(G)))
        assert np.array_equal(np.diag(G), np.abs(T).sum(axis=1))
        # rows are grouped by block, blocks contiguous
        for q, f in enumerate(first):
            assert (row_block[f:f + size[q]] == q).all()
        # the per-edge lists are the columns of T (at most 8 rows per edge)
        for e, lst in enumerate(edge_rows):
            assert 1 <= len(lst) <= 8
            col = np.zeros(nl)
            for r, s in lst:
                col[r] = s
            assert np.array_equal(col, T[:, e])
        # T^t M T is the dense operator, up to the float pairs' 48 bits and the
        # off-block part the construction drops (reported in `dropped`)
        err = np.abs(T.T @ M @ T - D).max() / np.abs(D).max()
        assert float(dropped) < 1e-6
        assert err < 64 * 2.0 ** -48 + 16 * float(dropped), (name, err, dropped)
