// Host-side (FP64) local operators for a curl-curl coefficient that is
// constant on every hexahedron (eq. 1 with a piecewise-constant alpha; the
// jumping coefficients of the concluding remarks).  The paper's smoother is
// unchanged: the same interior spaces (eq. SubdomainSpace), vertex spaces of
// discrete harmonic extensions (eq. vertex space) and edge spaces, each with
// its own local matrix.  Those matrices now depend on the coefficients of the
// cells they cover, so the subdomains / patches of a family are grouped by
// those values (bitwise equal cell coefficients give equal matrices) and one
// operator is built per group.  Coarse levels carry the mean of the 8 fine
// coefficients in each coarse hexahedron.
#include <algorithm>
#include <cstring>
#include <stdexcept>
#include <string>
#include <thread>
#include <unordered_map>

#include "kernels.cuh"
#include "tc_patch.cuh"

namespace ndmg {

std::vector<double> coarsen_cells(const std::vector<double>& a, int n) {
  const int c = n / 2;
  std::vector<double> out((size_t)c * c * c);
  for (int K = 0; K < c; ++K)
    for (int J = 0; J < c; ++J)
      for (int I = 0; I < c; ++I) {
        double s = 0.0;
        for (int dk = 0; dk < 2; ++dk)
          for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di)
              s += a[((size_t)(2 * K + dk) * n + (2 * J + dj)) * n + (2 * I + di)];
        out[((size_t)K * c + J) * c + I] = s / 8.0;
      }
  return out;
}

namespace {

// coefficients of the cells of member P of family f (box order, x fastest)
void member_cells(int n, const PatchFamily& f, const std::vector<double>& acell, int64_t P, double* out) {
  const int pa = (int)(P % f.np[0]) + f.p0[0];
  const int pb = (int)((P / f.np[0]) % f.np[1]) + f.p0[1];
  const int pc = (int)(P / ((int64_t)f.np[0] * f.np[1])) + f.p0[2];
  const int o[3] = {f.stride * pa - f.shift[0], f.stride * pb - f.shift[1], f.stride * pc - f.shift[2]};
  int q = 0;
  for (int ck = 0; ck < f.b[2]; ++ck)
    for (int cj = 0; cj < f.b[1]; ++cj)
      for (int ci = 0; ci < f.b[0]; ++ci)
        out[q++] = acell[((size_t)(o[2] + ck) * n + (o[1] + cj)) * n + (o[0] + ci)];
}

// group the members of f by their cell coefficients; reps: one member per group
void group_members(int n, const PatchFamily& f, const std::vector<double>& acell, int max_groups,
                   GroupedFamily* g, std::vector<std::vector<double>>* reps) {
  const int nc = f.b[0] * f.b[1] * f.b[2];
  const int64_t NP = (int64_t)f.np[0] * f.np[1] * f.np[2];
  std::unordered_map<std::string, int> seen;
  std::vector<double> cells(nc);
  std::string key(nc * sizeof(double), '\0');
  g->gid.assign((size_t)std::max<int64_t>(NP, 0), 0);
  reps->clear();
  for (int64_t P = 0; P < NP; ++P) {
    member_cells(n, f, acell, P, cells.data());
    std::memcpy(&key[0], cells.data(), key.size());
    auto it = seen.find(key);
    if (it == seen.end()) {
      if ((int)reps->size() >= max_groups)
        throw std::runtime_error("coefficient field: more than " + std::to_string(max_groups) +
                                 " distinct local problems on the " + std::to_string(n) + "^3 level");
      it = seen.emplace(key, (int)reps->size()).first;
      reps->push_back(cells);
    }
    g->gid[(size_t)P] = it->second;
  }
  g->ngroups = (int)reps->size();
}

// run body(group) for every group on the host's cores
template <typename F>
void for_groups(int ngroups, F&& body) {
  const int nt = std::max(1, std::min<int>(ngroups, (int)std::max(1u, std::thread::hardware_concurrency())));
  if (nt == 1) {
    for (int q = 0; q < ngroups; ++q) body(q);
    return;
  }
  std::vector<std::thread> pool;
  std::vector<std::string> errs(nt);
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([&, t] {
      try {
        for (int q = t; q < ngroups; q += nt) body(q);
      } catch (const std::exception& e) {
        errs[t] = e.what();
      }
    });
  for (auto& th : pool) th.join();
  for (auto& e : errs)
    if (!e.empty()) throw std::runtime_error(e);
}

}  // namespace

void build_field_ops(int n, double L, const std::vector<double>& acell, double beta, bool edge, int max_groups,
                     FieldOps* out, int lowp) {
  const double h = L / n;
  const int nc = n / 2;
  std::vector<std::vector<double>> reps;
  // interior spaces of the coarse elements (2x2x2 cells): 6x6 inverses
  {
    PatchFamily f{6, {2, 2, 2}, {nc, nc, nc}, {0, 0, 0}, {0, 0, 0}};
    GroupedFamily& g = out->bub;
    g.nloc = 6;
    group_members(n, f, acell, max_groups, &g, &reps);
    g.op.assign((size_t)g.ngroups * 36, 0.0);
    for_groups(g.ngroups, [&](int q) {
      bool ok = false;
      const std::vector<double> inv = spd_inverse(box_matrix_cells(Box{{2, 2, 2}}, h, reps[q].data(), beta), 6, &ok);
      if (!ok) throw std::runtime_error("interior-space matrix is not SPD");
      std::copy(inv.begin(), inv.end(), g.op.begin() + (size_t)q * 36);
    });
  }
  if (!edge) {
    // vertex patches (4x4x4 cells): dense 108x108 and Gram factor 108x60
    const PatchFamily f = vertex_family(n);
    GroupedFamily& g = out->vtx;
    g.nloc = 108;
    g.nG = 60;
    group_members(n, f, acell, max_groups, &g, &reps);
    g.op.assign((size_t)g.ngroups * 108 * 108, 0.0);
    g.W.assign((size_t)g.ngroups * 108 * 60, 0.0);
    std::vector<double> spec(g.ngroups, 0.0);
    for_groups(g.ngroups, [&](int q) {
      const Box vb{{4, 4, 4}};
      std::vector<double> D, W;
      int nG = 0;
      const std::vector<double> Ap = box_matrix_cells(vb, h, reps[q].data(), beta);
      patch_operator(vb, 2, Ap, &D, &W, &nG);
      if (nG != 60) throw std::runtime_error("unexpected vertex-patch split");
      std::copy(D.begin(), D.end(), g.op.begin() + (size_t)q * 108 * 108);
      std::copy(W.begin(), W.end(), g.W.begin() + (size_t)q * 108 * 60);
      if (lowp) spec[q] = tc_operand_spectral_max(W.data(), Ap, lowp == 2);
    });
    for (double v : spec) g.tc_spectral = std::max(g.tc_spectral, v);
    return;
  }
  // edge patches (2 cells along the coarse edge, 4 x 4 across): 42x42
  for (int d = 0; d < 3; ++d) {
    const PatchFamily f = edge_family(n, d);
    GroupedFamily& g = out->edge[d];
    g.nloc = 42;
    group_members(n, f, acell, max_groups, &g, &reps);
    g.op.assign((size_t)g.ngroups * 42 * 42, 0.0);
    for_groups(g.ngroups, [&](int q) {
      Box eb{{4, 4, 4}};
      eb.b[d] = 2;
      std::vector<double> D, W;
      int nG = 0;
      patch_operator(eb, 2, box_matrix_cells(eb, h, reps[q].data(), beta), &D, &W, &nG);
      if (nG != 18) throw std::runtime_error("unexpected edge-patch split");
      std::copy(D.begin(), D.end(), g.op.begin() + (size_t)q * 42 * 42);
    });
  }
}

std::vector<double> coarse_inverse_cells(int n0, double L, const std::vector<double>& acell, double beta) {
  const Box b{{n0, n0, n0}};
  const int N = (int)b.size();
  bool ok = false;
  std::vector<double> inv = spd_inverse(box_matrix_cells(b, L / n0, acell.data(), beta), N, &ok);
  if (!ok) throw std::runtime_error("coarsest operator is not SPD");
  return inv;
}

// members of each group in turn, cut into chunks of at most `pb` members
void group_chunks(const GroupedFamily& g, int pb, std::vector<int>* plist, std::vector<int>* chunks) {
  std::vector<int> count(g.ngroups + 1, 0);
  for (int q : g.gid) ++count[q + 1];
  for (int q = 0; q < g.ngroups; ++q) count[q + 1] += count[q];
  plist->assign(g.gid.size(), 0);
  std::vector<int> pos(count.begin(), count.end() - 1);
  for (size_t P = 0; P < g.gid.size(); ++P) (*plist)[pos[g.gid[P]]++] = (int)P;
  chunks->clear();
  for (int q = 0; q < g.ngroups; ++q)
    for (int s = count[q]; s < count[q + 1]; s += pb) {
      chunks->push_back(q);
      chunks->push_back(s);
      chunks->push_back(std::min(pb, count[q + 1] - s));
      chunks->push_back(0);
    }
}

}  // namespace ndmg
