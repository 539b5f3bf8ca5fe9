"""The library's host-side set-up for a curl-curl coefficient per hexahedron
(paper_2205_05840_gb300/csrc/field.cpp), built as a host program and checked
on the CPU against the oracle.

With a coefficient per cell the local problems of the smoother differ between
subdomains and patches; the set-up groups the members of each family (coarse
elements, vertex patches, edge patches) by the coefficients of the cells they
cover and builds one operator per group.  The test takes the groups, the
per-group operators, the families' geometry and the box numbering from the
library, scatters them onto the global mesh, and compares the additive
smoothers of eq. (Preconditioner P) and eq. (Preconditioner E) they define with
the oracle's smoother for the same field (local matrices taken from the
oracle's own assembly, grouped by equality); the coarse-grid coefficients and
the coarsest inverse are compared with the oracle's as well.  The program links
the CUDA translation units that hold the family geometry but runs on the host
only (no kernel is launched), so no GPU is needed."""
from __future__ import annotations

import os
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import hcurl, mg
from paper_2205_05840_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2205_05840_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>
#include "kernels.cuh"
using namespace ndmg;
static void wr(const std::string& p, const std::vector<double>& v) {
  FILE* f = fopen(p.c_str(), "wb"); fwrite(v.data(), sizeof(double), v.size(), f); fclose(f);
}
static std::vector<double> rd(const std::string& p) {
  FILE* f = fopen(p.c_str(), "rb"); fseek(f, 0, SEEK_END); long n = ftell(f); fseek(f, 0, SEEK_SET);
  std::vector<double> v(n / sizeof(double)); fread(v.data(), sizeof(double), v.size(), f); fclose(f); return v;
}
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
static std::vector<double> fam(const PatchFamily& f) {
  return {(double)f.nloc, (double)f.b[0], (double)f.b[1], (double)f.b[2], (double)f.np[0], (double)f.np[1],
          (double)f.np[2], (double)f.p0[0], (double)f.p0[1], (double)f.p0[2], (double)f.shift[0],
          (double)f.shift[1], (double)f.shift[2], (double)f.stride};
}
static void group(const std::string& p, const GroupedFamily& g) {
  wr(p + "_gid.bin", std::vector<double>(g.gid.begin(), g.gid.end()));
  wr(p + "_op.bin", g.op);
  // the kernels' work list: members group by group, chunks of at most 8
  std::vector<int> plist, chunks;
  group_chunks(g, 8, &plist, &chunks);
  wr(p + "_plist.bin", std::vector<double>(plist.begin(), plist.end()));
  wr(p + "_chunks.bin", std::vector<double>(chunks.begin(), chunks.end()));
}
int main(int argc, char** argv) {
  const std::string dir = argv[1];
  const int n = atoi(argv[2]), n0 = atoi(argv[3]);
  const double L = atof(argv[4]), beta = atof(argv[5]);
  const std::vector<double> a = rd(dir + "/acell.bin");
  for (int edge = 0; edge < 2; ++edge) {
    FieldOps ops;
    build_field_ops(n, L, a, beta, edge == 1, 8192, &ops, 0);
    if (edge == 0) {
      group(dir + "/bub", ops.bub);
      group(dir + "/vtx", ops.vtx);
      wr(dir + "/vtx_fam.bin", fam(vertex_family(n)));
    } else {
      for (int d = 0; d < 3; ++d) {
        group(dir + "/edge" + std::to_string(d), ops.edge[d]);
        wr(dir + "/edge" + std::to_string(d) + "_fam.bin", fam(edge_family(n, d)));
      }
    }
  }
  std::vector<double> ac = a;
  for (int m = n; m > n0; m /= 2) ac = coarsen_cells(ac, m);
  wr(dir + "/acell0.bin", ac);
  wr(dir + "/coarse_inv.bin", coarse_inverse_cells(n0, L, ac, beta));
  wr(dir + "/map_T.bin", box_map(Box{{2, 2, 2}}));
  wr(dir + "/map_V.bin", box_map(Box{{4, 4, 4}}));
  for (int d = 0; d < 3; ++d) {
    Box eb{{4, 4, 4}};
    eb.b[d] = 2;
    wr(dir + "/map_E" + std::to_string(d) + ".bin", box_map(eb));
  }
  return 0;
}
"""

SOURCES = ["field.cpp", "setup.cpp", "kernels.cu", "tc_patch.cu"]


@pytest.fixture(scope="module")
def driver(host_build, tmp_path_factory):
    return host_build(DRIVER, SOURCES), str(tmp_path_factory.mktemp("field_host"))


def _run(driver, tag, acell, n, n0, L, beta):
    exe, d = driver
    out = os.path.join(d, tag)
    os.makedirs(out, exist_ok=True)
    np.asarray(acell, dtype=np.float64).tofile(os.path.join(out, "acell.bin"))
    subprocess.run([exe, out, str(n), str(n0), repr(L), repr(beta)], check=True, capture_output=True)
    rd = lambda name: np.fromfile(os.path.join(out, name + ".bin"), dtype=np.float64)  # noqa: E731
    return rd


def _global(n, box_map, origin):
    d, i, j, k = box_map.T
    return hcurl.edge_index(n, d, origin[0] + i, origin[1] + j, origin[2] + k)


def _members(fam):
    """Box origins (node coordinates) of the members of a family, member P
    with x fastest, as the library lays out a family."""
    f = fam.astype(int)
    b, npa, p0, shift, stride = f[1:4], f[4:7], f[7:10], f[10:13], f[13]
    out = []
    for P in range(int(np.prod(npa))):
        p = np.array([P % npa[0], (P // npa[0]) % npa[1], P // (npa[0] * npa[1])])
        out.append(stride * (p + p0) - shift)
    return b, out


def _scatter(M, n, rd, name, nloc, box_map, origins):
    gid = rd(name + "_gid").astype(int)
    op = rd(name + "_op").reshape(-1, nloc, nloc)
    assert gid.size == len(origins) and gid.max() + 1 == op.shape[0]
    for P, o in enumerate(origins):
        idx = _global(n, box_map, o)
        assert (idx >= 0).all()
        M[np.ix_(idx, idx)] += op[gid[P]]


def _field_smoother(n, rd, kind):
    N = hcurl.num_edges(n)
    M = np.zeros((N, N))
    nc = n // 2
    # coarse elements: cells [2c, 2c + 2), x fastest
    elems = [2 * np.array([c % nc, (c // nc) % nc, c // (nc * nc)]) for c in range(nc ** 3)]
    _scatter(M, n, rd, "bub", 6, rd("map_T").reshape(-1, 4).astype(int), elems)
    if kind == "vertex":
        b, origins = _members(rd("vtx_fam"))
        assert tuple(b) == (4, 4, 4)
        _scatter(M, n, rd, "vtx", 108, rd("map_V").reshape(-1, 4).astype(int), origins)
    else:
        for d in range(3):
            b, origins = _members(rd(f"edge{d}_fam"))
            assert b[d] == 2 and sorted(b) == [2, 4, 4]
            _scatter(M, n, rd, f"edge{d}", 42, rd(f"map_E{d}").reshape(-1, 4).astype(int), origins)
    return M


FIELDS = {
    "inclusion": lambda n: inputs.inclusion_field(n, 1.0, 10.0),
    "checker": lambda n: inputs.checker_field(n, 2, 1.0, 100.0),
    "random": lambda n: inputs.random_field(n, 3, 0.1, 10.0),
}


@pytest.mark.parametrize("field", sorted(FIELDS))
@pytest.mark.parametrize("n,n0,L,beta", [(8, 2, 1.0, 1.0), (8, 4, 1.3, 2.9)])
def test_field_setup_reproduces_the_oracle_smoothers(driver, field, n, n0, L, beta):
    a = FIELDS[field](n)
    rd = _run(driver, f"{field}_{n}_{n0}_{L}", a, n, n0, L, beta)
    A = hcurl.assemble_field(n, L, a, beta)
    rng = np.random.default_rng(4)
    R = rng.standard_normal((A.shape[0], 5))
    for kind, eta in (("vertex", 1.0 / 9.0), ("edge", 1.0 / 13.0)):
        S = mg.Smoother(A, n, kind, varying=True)
        assert S.eta == eta
        want = np.stack([S.apply(R[:, c]) for c in range(R.shape[1])], axis=1)
        got = eta * (_field_smoother(n, rd, kind) @ R)
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err < 1e-10, (kind, err)
    # coarse-grid coefficients (8-cell means per level) and the coarsest inverse
    ac, m = np.asarray(a, dtype=float), n
    while m > n0:
        ac = mg.coarsen_field(ac, m)
        m //= 2
    assert np.abs(rd("acell0") - ac).max() <= 1e-15 * np.abs(ac).max()
    A0 = hcurl.assemble_field(n0, L, ac, beta).toarray()
    inv = rd("coarse_inv").reshape(A0.shape)
    assert np.abs(inv - sla.inv(A0)).max() <= 1e-10 * np.abs(inv).max()


def test_field_groups_follow_the_cell_coefficients(driver):
    # a constant field: one group per family; one cell changed: only the
    # members covering that cell leave the common group
    n = 8
    a = np.ones(n ** 3)
    rd = _run(driver, "const", a, n, 2, 1.0, 1.0)
    assert (rd("bub_gid") == 0).all() and (rd("vtx_gid") == 0).all()
    a[(3 * n + 4) * n + 5] = 7.0          # cell (5, 4, 3)
    rd = _run(driver, "one_cell", a, n, 2, 1.0, 1.0)
    for name, fam, b in (("vtx", rd("vtx_fam"), 4),):
        _, origins = _members(fam)
        gid = rd(name + "_gid").astype(int)
        for o, g in zip(origins, gid):
            covers = all(o[ax] <= (5, 4, 3)[ax] < o[ax] + b for ax in range(3))
            assert (g != 0) == covers, (o, g)
    gid_b = rd("bub_gid").astype(int)
    nc = n // 2
    for c in range(nc ** 3):
        o = 2 * np.array([c % nc, (c // nc) % nc, c // (nc * nc)])
        covers = all(o[ax] <= (5, 4, 3)[ax] < o[ax] + 2 for ax in range(3))
        assert (gid_b[c] != 0) == covers


@pytest.mark.parametrize("field", sorted(FIELDS))
def test_field_work_lists_cover_every_member_once(driver, field):
    # the grouped kernels walk chunks {group, first, count} of the member list
    # (members listed group by group): every member exactly once, a chunk
    # holds at most 8 members of one group
    n = 8
    rd = _run(driver, f"chunks_{field}", FIELDS[field](n), n, 2, 1.0, 1.0)
    for name in ("bub", "vtx", "edge0", "edge1", "edge2"):
        gid = rd(name + "_gid").astype(int)
        plist = rd(name + "_plist").astype(int)
        chunks = rd(name + "_chunks").astype(int).reshape(-1, 4)
        assert sorted(plist) == list(range(gid.size))
        covered = []
        for q, first, count, pad in chunks:
            assert 1 <= count <= 8 and pad == 0
            members = plist[first:first + count]
            assert (gid[members] == q).all()
            covered.extend(members)
        assert sorted(covered) == list(range(gid.size))
