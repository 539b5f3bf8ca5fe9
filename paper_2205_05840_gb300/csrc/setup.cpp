// Host-side (FP64) construction of the local operators of the smoother and of
// the coarsest solve.  Everything here runs once per (n, L, alpha, beta).
//
// Element matrices of the lowest-order hexahedral Nedelec element (Sec. 2,
// eq. nedlec form / NDdof) on a cube of side h, written in closed form.  With
// l_0(t) = 1 - t/h, l_1(t) = t/h, int_0^h l_a l_c = h m_ac,
// m = [[1/3, 1/6], [1/6, 1/3]], l_a' = s_a / h, s = (-1, +1), and the basis
// function of the edge along axis d whose start vertex sits at offset a on
// axis d+1 and b on axis d+2 (cyclic) equal to l_a l_b e_d:
//   mass            M = h^3 m_{a a'} m_{b b'}                     (same axis)
//   curl-curl       K = h (m_{a a'} s_b s_b' + s_a s_a' m_{b b'})  (same axis)
//                   K = -h s_a s_b' m_{b a'}   (second edge along axis d+1)
// The local spaces of Sec. 3.2 are boxes of cells with only the edges in the
// box's relative interior, which is the same numbering as the global mesh.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "ndmg_internal.h"

namespace ndmg {

int64_t Box::index(int d, int i, int j, int k) const {
  const int p[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    if (a == d) {
      if (p[a] < 0 || p[a] >= b[a]) return -1;
    } else {
      if (p[a] < 1 || p[a] > b[a] - 1) return -1;
    }
  }
  const int bx = b[0], by = b[1];
  if (d == 0) return ((int64_t)(k - 1) * (by - 1) + (j - 1)) * bx + i;
  if (d == 1) return count(0) + ((int64_t)(k - 1) * by + j) * (bx - 1) + (i - 1);
  return count(0) + count(1) + ((int64_t)k * (by - 1) + (j - 1)) * (bx - 1) + (i - 1);
}

namespace {

const double kM[2][2] = {{1.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 1.0 / 3.0}};
const double kS[2] = {-1.0, 1.0};

struct LocalEdge {
  int d, a, b;
};

LocalEdge local_edge(int e) { return LocalEdge{e / 4, e % 2, (e / 2) % 2}; }

// 12x12 element matrix alpha K + beta M of one cube of side h.
void element_matrix(double h, double alpha, double beta, double out[12][12]) {
  for (int p = 0; p < 12; ++p) {
    for (int q = 0; q < 12; ++q) {
      LocalEdge e1 = local_edge(p), e2 = local_edge(q);
      double kv = 0.0, mv = 0.0;
      if (e1.d == e2.d) {
        mv = h * h * h * kM[e1.a][e2.a] * kM[e1.b][e2.b];
        kv = h * (kM[e1.a][e2.a] * kS[e1.b] * kS[e2.b] + kS[e1.a] * kS[e2.a] * kM[e1.b][e2.b]);
      } else if (e2.d == (e1.d + 1) % 3) {
        kv = -h * kS[e1.a] * kS[e2.b] * kM[e1.b][e2.a];
      } else {
        kv = -h * kS[e2.a] * kS[e1.b] * kM[e2.b][e1.a];
      }
      out[p][q] = alpha * kv + beta * mv;
    }
  }
}

}  // namespace

// Sum of the element matrices of the box's cells over its interior edges;
// elem(cell) gives the 12x12 matrix of cell (ci, cj, ck), cell = (ck by + cj) bx + ci.
template <typename Elem>
static std::vector<double> assemble_box(const Box& box, Elem&& elem) {
  const int64_t N = box.size();
  std::vector<double> A((size_t)(N * N), 0.0);
  int64_t gid[12];
  for (int ck = 0; ck < box.b[2]; ++ck)
    for (int cj = 0; cj < box.b[1]; ++cj)
      for (int ci = 0; ci < box.b[0]; ++ci) {
        const int c[3] = {ci, cj, ck};
        const double(&E)[12][12] = elem((ck * box.b[1] + cj) * box.b[0] + ci);
        for (int e = 0; e < 12; ++e) {
          LocalEdge le = local_edge(e);
          int p[3] = {c[0], c[1], c[2]};
          p[(le.d + 1) % 3] += le.a;
          p[(le.d + 2) % 3] += le.b;
          gid[e] = box.index(le.d, p[0], p[1], p[2]);
        }
        for (int e = 0; e < 12; ++e) {
          if (gid[e] < 0) continue;
          for (int f = 0; f < 12; ++f) {
            if (gid[f] < 0) continue;
            A[(size_t)(gid[e] * N + gid[f])] += E[e][f];
          }
        }
      }
  return A;
}

std::vector<double> box_matrix(const Box& box, double h, double alpha, double beta) {
  double E[12][12];
  element_matrix(h, alpha, beta, E);
  return assemble_box(box, [&](int) -> const double(&)[12][12] { return E; });
}

std::vector<double> box_matrix_cells(const Box& box, double h, const double* acell, double beta) {
  double Kh[12][12], Mh[12][12], E[12][12];
  element_matrix(h, 1.0, 0.0, Kh);
  element_matrix(h, 0.0, 1.0, Mh);
  return assemble_box(box, [&](int c) -> const double(&)[12][12] {
    for (int p = 0; p < 12; ++p)
      for (int q = 0; q < 12; ++q) E[p][q] = acell[c] * Kh[p][q] + beta * Mh[p][q];
    return E;
  });
}

bool cholesky(std::vector<double>& a, int n) {
  for (int j = 0; j < n; ++j) {
    double s = a[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= a[(size_t)j * n + k] * a[(size_t)j * n + k];
    if (!(s > 0.0)) return false;
    const double d = std::sqrt(s);
    a[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = a[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= a[(size_t)i * n + k] * a[(size_t)j * n + k];
      a[(size_t)i * n + j] = t / d;
    }
    for (int i = 0; i < j; ++i) a[(size_t)i * n + j] = 0.0;
  }
  return true;
}

// solve L y = b in place (L lower triangular, row-major)
void forward_solve(const std::vector<double>& Lm, int n, double* b) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= Lm[(size_t)i * n + k] * b[k];
    b[i] = s / Lm[(size_t)i * n + i];
  }
}

// solve L L^t x = b in place
void chol_solve(const std::vector<double>& Lm, int n, double* b) {
  forward_solve(Lm, n, b);
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= Lm[(size_t)k * n + i] * b[k];
    b[i] = s / Lm[(size_t)i * n + i];
  }
}

std::vector<double> spd_inverse(const std::vector<double>& a, int n, bool* ok) {
  std::vector<double> Lm = a;
  *ok = cholesky(Lm, n);
  if (!*ok) return {};
  std::vector<double> inv((size_t)n * n, 0.0), e(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) e[i] = (i == c) ? 1.0 : 0.0;
    chol_solve(Lm, n, e.data());
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = e[i];
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      const double m = 0.5 * (inv[(size_t)i * n + j] + inv[(size_t)j * n + i]);
      inv[(size_t)i * n + j] = inv[(size_t)j * n + i] = m;
    }
  return inv;
}

// J_D A_D^{-1} J_D^t for the discrete-harmonic patch space of a box of
// cells (Sec. 3.2, eq. vertex space / edge space): the box's edges split into
// the interiors of its s x s x s subdomains (I) and the rest (G); with
// S = A_GG - A_GI A_II^{-1} A_IG = R R^t and H = [-A_II^{-1} A_IG ; I],
// W = H R^{-t} and D = W W^t (= A_p^{-1} - sum_T J_T A_T^{-1} J_T^t).
// Ap: the assembled matrix of the box (its own canonical order); the
// subdomains' interior-space inverses (its diagonal blocks on I) serve the
// self-check.  D may be null (large patches: only W).
void patch_operator(const Box& pb, int s, const std::vector<double>& Ap, std::vector<double>* D,
                    std::vector<double>* W, int* n_interface) {
  const int np = (int)pb.size();
  // the interior spaces of the subdomains inside the box, each in its s-box
  // order; Bblk = sum_T J_T A_T^{-1} J_T^t restricted to the box
  const Box sb{{s, s, s}};
  const int mT = (int)sb.size();
  std::vector<int> isB(np, 0);
  std::vector<double> Bblk((size_t)np * np, 0.0);
  std::vector<int> ids(mT);
  for (int sr = 0; sr < pb.b[2] / s; ++sr)
    for (int sq = 0; sq < pb.b[1] / s; ++sq)
      for (int sp = 0; sp < pb.b[0] / s; ++sp) {
        const int o[3] = {s * sp, s * sq, s * sr};
        for (int d = 0; d < 3; ++d)
          for (int k = 0; k < s; ++k)
            for (int j = 0; j < s; ++j)
              for (int i = 0; i < s; ++i) {
                const int64_t l = sb.index(d, i, j, k);
                if (l >= 0) ids[l] = (int)pb.index(d, o[0] + i, o[1] + j, o[2] + k);
              }
        // this subdomain's interior-space inverse (its block of A_p)
        std::vector<double> AT((size_t)mT * mT);
        for (int a = 0; a < mT; ++a)
          for (int b = 0; b < mT; ++b) AT[(size_t)a * mT + b] = Ap[(size_t)ids[a] * np + ids[b]];
        bool ok = false;
        const std::vector<double> AinvT = spd_inverse(AT, mT, &ok);
        if (!ok) throw std::runtime_error("interior-space block is not SPD");
        for (int a = 0; a < mT; ++a) {
          isB[ids[a]] = 1;
          for (int b = 0; b < mT; ++b) Bblk[(size_t)ids[a] * np + ids[b]] = AinvT[(size_t)a * mT + b];
        }
      }

  // Gram factor through the Schur complement on the interface edges
  std::vector<int> I, G;
  for (int e = 0; e < np; ++e) (isB[e] ? I : G).push_back(e);
  const int nI = (int)I.size(), nG = (int)G.size();
  *n_interface = nG;
  std::vector<double> AII((size_t)nI * nI), AIG((size_t)nI * nG), AGG((size_t)nG * nG);
  for (int a = 0; a < nI; ++a)
    for (int b = 0; b < nI; ++b) AII[(size_t)a * nI + b] = Ap[(size_t)I[a] * np + I[b]];
  for (int a = 0; a < nI; ++a)
    for (int b = 0; b < nG; ++b) AIG[(size_t)a * nG + b] = Ap[(size_t)I[a] * np + G[b]];
  for (int a = 0; a < nG; ++a)
    for (int b = 0; b < nG; ++b) AGG[(size_t)a * nG + b] = Ap[(size_t)G[a] * np + G[b]];
  // Every step below uses triangular solves with Cholesky factors, never an
  // explicit inverse: for alpha / (beta h^2) ~ 1e4 and beyond the patch matrix
  // has cond ~ 1e6, and explicit inverses lose three more digits than solves.
  std::vector<double> LII = AII;
  if (!cholesky(LII, nI)) throw std::runtime_error("bubble block is not SPD");
  // X = A_II^{-1} A_IG (nI x nG), column by column
  std::vector<double> X((size_t)nI * nG, 0.0), col(nI);
  for (int b = 0; b < nG; ++b) {
    for (int a = 0; a < nI; ++a) col[a] = AIG[(size_t)a * nG + b];
    chol_solve(LII, nI, col.data());
    for (int a = 0; a < nI; ++a) X[(size_t)a * nG + b] = col[a];
  }
  // Schur complement S = A_GG - A_GI X, symmetrised
  std::vector<double> S = AGG;
  for (int a = 0; a < nG; ++a)
    for (int b = 0; b < nG; ++b) {
      double sdot = 0.0;
      for (int k = 0; k < nI; ++k) sdot += AIG[(size_t)k * nG + a] * X[(size_t)k * nG + b];
      S[(size_t)a * nG + b] -= sdot;
    }
  for (int a = 0; a < nG; ++a)
    for (int b = 0; b < a; ++b) {
      const double m = 0.5 * (S[(size_t)a * nG + b] + S[(size_t)b * nG + a]);
      S[(size_t)a * nG + b] = S[(size_t)b * nG + a] = m;
    }
  std::vector<double> R = S;
  if (!cholesky(R, nG)) throw std::runtime_error("Schur complement is not SPD");
  // W^t = R^{-1} H^t with H = [-X ; I] (patch order): forward substitution on
  // each of the np columns of H^t
  (*W).assign((size_t)np * nG, 0.0);
  std::vector<int> pos(np);
  for (int a = 0; a < nI; ++a) pos[I[a]] = a;
  for (int g = 0; g < nG; ++g) pos[G[g]] = g;
  std::vector<double> ht(nG);
  for (int e = 0; e < np; ++e) {
    if (isB[e]) {
      const int a = pos[e];
      for (int c = 0; c < nG; ++c) ht[c] = -X[(size_t)a * nG + c];
    } else {
      const int g = pos[e];
      for (int c = 0; c < nG; ++c) ht[c] = (c == g) ? 1.0 : 0.0;
    }
    forward_solve(R, nG, ht.data());
    for (int c = 0; c < nG; ++c) (*W)[(size_t)e * nG + c] = ht[c];
  }
  // The dense operator used by the CUDA-core kernels is D = W W^t as well:
  // forming A_p^{-1} - Bblk instead would cancel the large bubble entries and
  // lose ~cond(A_p) digits.  Self-check with a residual that stays well
  // scaled: A_p (W W^t + Bblk) = I (Sec. 3.2: the patch space is the direct
  // sum of the subdomain interior spaces and the a-orthogonal vertex space),
  // on every column for small patches and on a spread of columns for large ones.
  if (D) {
    (*D).assign((size_t)np * np, 0.0);
    for (int a = 0; a < np; ++a)
      for (int b = 0; b < np; ++b) {
        double sdot = 0.0;
        for (int c = 0; c < nG; ++c) sdot += (*W)[(size_t)a * nG + c] * (*W)[(size_t)b * nG + c];
        (*D)[(size_t)a * np + b] = sdot;
      }
  }
  const int step = np <= 200 ? 1 : 37;
  std::vector<double> pcol(np), tmp(nG);
  double err = 0.0;
  for (int b = 0; b < np; b += step) {
    // pcol = (W W^t + Bblk) e_b
    for (int c = 0; c < nG; ++c) tmp[c] = (*W)[(size_t)b * nG + c];
    for (int a = 0; a < np; ++a) {
      double sdot = Bblk[(size_t)a * np + b];
      for (int c = 0; c < nG; ++c) sdot += (*W)[(size_t)a * nG + c] * tmp[c];
      pcol[a] = sdot;
    }
    for (int a = 0; a < np; ++a) {
      double sdot = 0.0;
      for (int c = 0; c < np; ++c) sdot += Ap[(size_t)a * np + c] * pcol[c];
      err = std::fmax(err, std::fabs(sdot - (a == b ? 1.0 : 0.0)));
    }
  }
  // rounding grows like cond(A_p)^2 eps here (cond ~ alpha / (beta h^2));
  // an indexing mistake gives O(1), so 1e-3 separates the two up to n ~ 1000
  if (!(err <= 1e-3)) throw std::runtime_error("Gram factor does not reproduce the patch operator");
}


void build_local_ops(int n, double L, double alpha, double beta, LocalOps* out, int s) {
  const double h = L / n;
  out->n = n;
  out->h = h;
  out->s = s;
  bool ok = false;
  // interior space N_h^T of one subdomain (s x s x s cells; s = 2: a coarse
  // element with 6 interior edges)
  const Box bub{{s, s, s}};
  out->mT = (int)bub.size();
  std::vector<double> AT = box_matrix(bub, h, alpha, beta);
  out->AinvT = spd_inverse(AT, out->mT, &ok);
  if (!ok) throw std::runtime_error("interior-space matrix is not SPD");
  // vertex patch: the 2s x 2s x 2s cells around a subdomain vertex; 108
  // interior edges and 60 on the interface for s = 2 (eq. vertex space),
  // 1176 and 312 for s = 4
  const Box vb{{2 * s, 2 * s, 2 * s}};
  out->mV = (int)vb.size();
  int nG = 0;
  patch_operator(vb, s, box_matrix(vb, h, alpha, beta), s == 2 ? &out->Dv : nullptr, &out->Wv, &nG);
  out->nG = nG;
  if (nG != out->mV - 8 * out->mT) throw std::runtime_error("unexpected vertex-patch split");
  if (s != 2) return;
  // edge patches: 2 cells along the coarse edge, 4 x 4 across, 42 interior
  // edges, 18 on the interface (eq. edge space); one operator per direction
  for (int d = 0; d < 3; ++d) {
    Box eb{{4, 4, 4}};
    eb.b[d] = 2;
    std::vector<double> We;
    patch_operator(eb, 2, box_matrix(eb, h, alpha, beta), &out->De[d], &We, &nG);
    if (nG != 18) throw std::runtime_error("unexpected edge-patch split");
  }
}

std::vector<double> coarse_inverse(int n0, double L, double alpha, double beta) {
  const Box b{{n0, n0, n0}};
  const int N = (int)b.size();
  std::vector<double> A = box_matrix(b, L / n0, alpha, beta);
  bool ok = false;
  std::vector<double> inv = spd_inverse(A, N, &ok);
  if (!ok) throw std::runtime_error("coarsest operator is not SPD");
  return inv;
}

}  // namespace ndmg
