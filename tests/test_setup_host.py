"""The library's host-side level set-up (paper_2205_05840_gb300/csrc/setup.cpp),
compiled as host C++ and checked on the CPU against the oracle.

The set-up forms the local operators every smoother kernel applies: the 6 x 6
inverse of the interior-space matrix A_T of a coarse element, the 108 x 108
vertex-patch operator J_V A_V^{-1} J_V^t (Sec. 3.2, eq. vertex space) with its
Gram factor W (108 x 60), the three 42 x 42 edge-patch operators (Sec. 3.3)
and the dense inverse of the coarsest operator (Fig. 1, k = 0).  It reaches
them from closed-form element matrices and Cholesky solves on each box of
cells, in the box's own edge numbering; the oracle reaches the same operators
from quadrature, a sparse global assembly and Schur complements on global edge
index sets.  The test scatters the set-up's local operators onto a global mesh
through the box numbering the set-up itself reports (Box::index), forms the
additive smoothers M^{-1} of eq. (Preconditioner P) and eq. (Preconditioner E)
from them, and compares their action with the oracle's on random vectors; the
coarsest inverse is compared with the inverse of the oracle's assembled
matrix.  No GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import hcurl, mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2205_05840_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>
#include "ndmg_internal.h"
using namespace ndmg;
static void wr(const std::string& p, const std::vector<double>& v) {
  FILE* f = fopen(p.c_str(), "wb"); fwrite(v.data(), sizeof(double), v.size(), f); fclose(f);
}
// (d, i, j, k) of every interior edge of a box, in the box's own numbering
static std::vector<double> box_map(const Box& b) {
  std::vector<double> m(4 * b.size(), -1.0);
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k <= b.b[2]; ++k)
      for (int j = 0; j <= b.b[1]; ++j)
        for (int i = 0; i <= b.b[0]; ++i) {
          const int64_t e = b.index(d, i, j, k);
          if (e < 0) continue;
          m[4 * e] = d; m[4 * e + 1] = i; m[4 * e + 2] = j; m[4 * e + 3] = k;
        }
  return m;
}
int main(int argc, char** argv) {
  const std::string dir = argv[1];
  const int n = atoi(argv[2]), n0 = atoi(argv[3]);
  const double L = atof(argv[4]), alpha = atof(argv[5]), beta = atof(argv[6]);
  const int s = argc > 7 ? atoi(argv[7]) : 2;
  LocalOps ops;
  build_local_ops(n, L, alpha, beta, &ops, s);
  if (s != 2) {  // subdomains of s^3 cells: interior inverses and the Gram factor only
    wr(dir + "/AinvT.bin", ops.AinvT);
    wr(dir + "/Wv.bin", ops.Wv);
    wr(dir + "/map_T.bin", box_map(Box{{s, s, s}}));
    wr(dir + "/map_V.bin", box_map(Box{{2 * s, 2 * s, 2 * s}}));
    printf("%d %d %d\n", ops.mT, ops.mV, ops.nG);
    return 0;
  }
  wr(dir + "/AinvT.bin", ops.AinvT);
  wr(dir + "/Dv.bin", ops.Dv);
  wr(dir + "/Wv.bin", ops.Wv);
  for (int d = 0; d < 3; ++d) wr(dir + "/De" + std::to_string(d) + ".bin", ops.De[d]);
  wr(dir + "/coarse_inv.bin", coarse_inverse(n0, L, alpha, beta));
  wr(dir + "/map_T.bin", box_map(Box{{2, 2, 2}}));
  wr(dir + "/map_V.bin", box_map(Box{{4, 4, 4}}));
  for (int d = 0; d < 3; ++d) {
    Box eb{{4, 4, 4}};
    eb.b[d] = 2;
    wr(dir + "/map_E" + std::to_string(d) + ".bin", box_map(eb));
  }
  printf("%d %d %d\n", ops.mT, ops.mV, ops.nG);
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("no host C++ compiler or CUDA headers")
    d = str(tmp_path_factory.mktemp("setup_host"))
    src = os.path.join(d, "drv.cpp")
    with open(src, "w") as fh:
        fh.write(DRIVER)
    exe = os.path.join(d, "drv")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, src, os.path.join(CSRC, "setup.cpp"),
                    "-o", exe], check=True)
    return exe, d


def _run(driver, n, n0, L, alpha, beta):
    exe, d = driver
    out = os.path.join(d, f"run_{n}_{n0}_{alpha}")
    os.makedirs(out, exist_ok=True)
    res = subprocess.run([exe, out, str(n), str(n0), repr(L), repr(alpha), repr(beta)], check=True,
                         capture_output=True, text=True)
    mT, mV, nG = map(int, res.stdout.split())
    rd = lambda name: np.fromfile(os.path.join(out, name + ".bin"), dtype=np.float64)  # noqa: E731
    ops = {"mT": mT, "mV": mV, "nG": nG,
           "AinvT": rd("AinvT").reshape(mT, mT), "Dv": rd("Dv").reshape(mV, mV), "Wv": rd("Wv").reshape(mV, nG),
           "De": [rd(f"De{k}").reshape(42, 42) for k in range(3)], "coarse_inv": rd("coarse_inv"),
           "map_T": rd("map_T").reshape(-1, 4).astype(int), "map_V": rd("map_V").reshape(-1, 4).astype(int),
           "map_E": [rd(f"map_E{k}").reshape(-1, 4).astype(int) for k in range(3)]}
    return ops


def _run_s(driver, n, L, alpha, beta, s):
    exe, d = driver
    out = os.path.join(d, f"run_s{s}_{n}_{alpha}")
    os.makedirs(out, exist_ok=True)
    res = subprocess.run([exe, out, str(n), "2", repr(L), repr(alpha), repr(beta), str(s)], check=True,
                         capture_output=True, text=True)
    mT, mV, nG = map(int, res.stdout.split())
    rd = lambda name: np.fromfile(os.path.join(out, name + ".bin"), dtype=np.float64)  # noqa: E731
    return {"mT": mT, "mV": mV, "nG": nG, "AinvT": rd("AinvT").reshape(mT, mT), "Wv": rd("Wv").reshape(mV, nG),
            "map_T": rd("map_T").reshape(-1, 4).astype(int), "map_V": rd("map_V").reshape(-1, 4).astype(int)}


def _global(n, box_map, origin):
    """Global edge indices of a box's edges (its own numbering) placed with
    its lowest node at `origin` (node coordinates)."""
    d, i, j, k = box_map.T
    return hcurl.edge_index(n, d, origin[0] + i, origin[1] + j, origin[2] + k)


def _setup_smoother(n, ops, kind):
    """eta-free additive operator sum_T J_T A_T^{-1} J_T^t + sum_D J_D op_D
    J_D^t from the set-up's local operators, as a dense matrix."""
    N = hcurl.num_edges(n)
    M = np.zeros((N, N))
    nc = n // 2

    def add(op, idx):
        assert (idx >= 0).all()
        M[np.ix_(idx, idx)] += op

    for c in np.ndindex(nc, nc, nc):           # coarse elements: cells [2c, 2c + 2)
        add(ops["AinvT"], _global(n, ops["map_T"], 2 * np.array(c[::-1])))
    if kind == "vertex":                       # interior coarse vertices v: cells [2v - 2, 2v + 2)
        for v in np.ndindex(nc - 1, nc - 1, nc - 1):
            v = np.array(v[::-1]) + 1
            add(ops["Dv"], _global(n, ops["map_V"], 2 * v - 2))
    else:                                      # interior coarse edges along d
        for d in range(3):
            ext = [nc if a == d else nc - 1 for a in range(3)]
            for v in np.ndindex(*ext[::-1]):
                v = np.array(v[::-1]) + (np.arange(3) != d)   # transverse coarse nodes 1 .. nc - 1
                o = 2 * v - 2                                  # cells [2v - 2, 2v + 2) across the edge,
                o[d] = 2 * v[d]                                # [2v, 2v + 2) along it
                add(ops["De"][d], _global(n, ops["map_E"][d], o))
    return M


@pytest.mark.parametrize("n,n0,L,alpha,beta", [(4, 2, 1.0, 1.0, 1.0), (8, 2, 1.3, 0.37, 2.9),
                                               (8, 4, 1.0, 100.0, 1.0), (12, 3, 1.0, 0.01, 1.0)])
def test_setup_local_operators_reproduce_the_oracle_smoothers(driver, n, n0, L, alpha, beta):
    ops = _run(driver, n, n0, L, alpha, beta)
    assert (ops["mT"], ops["mV"], ops["nG"]) == (6, 108, 60)
    # the Gram factor reproduces the vertex-patch operator
    assert np.abs(ops["Wv"] @ ops["Wv"].T - ops["Dv"]).max() <= 1e-9 * np.abs(ops["Dv"]).max()
    A = hcurl.assemble(n, L, alpha, beta)
    rng = np.random.default_rng(11)
    R = rng.standard_normal((A.shape[0], 6))
    for kind, eta in (("vertex", 1.0 / 9.0), ("edge", 1.0 / 13.0)):
        Msetup = eta * _setup_smoother(n, ops, kind)
        S = mg.Smoother(A, n, kind)
        assert S.eta == eta
        want = np.stack([S.apply(R[:, c]) for c in range(R.shape[1])], axis=1)
        got = Msetup @ R
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err < 1e-10, (kind, err)
        # and the whole operator is symmetric
        assert np.abs(Msetup - Msetup.T).max() <= 1e-12 * np.abs(Msetup).max()


@pytest.mark.parametrize("n0,L,alpha,beta", [(2, 1.0, 1.0, 1.0), (3, 1.3, 0.37, 2.9), (4, 1.0, 100.0, 1.0)])
def test_setup_coarsest_inverse_is_the_inverse_of_the_assembled_operator(driver, n0, L, alpha, beta):
    ops = _run(driver, 2 * n0, n0, L, alpha, beta)
    A0 = hcurl.assemble(n0, L, alpha, beta).toarray()
    inv = ops["coarse_inv"].reshape(A0.shape)
    ref = sla.inv(A0)
    assert np.abs(inv - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.abs(inv @ A0 - np.eye(A0.shape[0])).max() <= 1e-10


def test_setup_box_numbering_is_the_canonical_layout(driver):
    # the box numbering the set-up uses for its local operators equals the
    # canonical global numbering of an n^3 mesh when the box is the mesh
    ops = _run(driver, 4, 2, 1.0, 1.0, 1.0)
    m = ops["map_V"]            # a 4 x 4 x 4 box
    assert (_global(4, m, np.zeros(3, dtype=int)) == np.arange(hcurl.num_edges(4))).all()


@pytest.mark.parametrize("alpha", [1.0, 30.0])
def test_setup_subdomain4_operators_reproduce_the_oracle_smoother(driver, alpha):
    # subdomains of 4^3 cells: 108 x 108 interior-space inverses and the
    # Gram factor W (1176 x 312) of the 8^3-cell vertex patches, applied as
    # W (W^t r) patch by patch (the dense 1176^2 operator is never formed)
    n, s, L, beta = 16, 4, 1.0, 1.0
    ops = _run_s(driver, n, L, alpha, beta, s)
    assert (ops["mT"], ops["mV"], ops["nG"]) == (108, 1176, 312)
    A = hcurl.assemble(n, L, alpha, beta)
    R = np.random.default_rng(12).standard_normal((A.shape[0], 4))
    got = np.zeros_like(R)
    nc = n // s
    for c in np.ndindex(nc, nc, nc):                 # subdomains: cells [4c, 4c + 4)
        idx = _global(n, ops["map_T"], s * np.array(c[::-1]))
        assert (idx >= 0).all()
        got[idx] += ops["AinvT"] @ R[idx]
    for v in np.ndindex(nc - 1, nc - 1, nc - 1):     # interior subdomain vertices: cells [4v - 4, 4v + 4)
        idx = _global(n, ops["map_V"], s * (np.array(v[::-1]) + 1) - s)
        assert (idx >= 0).all()
        got[idx] += ops["Wv"] @ (ops["Wv"].T @ R[idx])
    S = mg.Smoother(A, n, "vertex", s=s)
    want = np.stack([S.apply(R[:, c]) for c in range(R.shape[1])], axis=1) / S.eta
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 1e-10, err
