// The smallest levels of the float V-cycle (Fig. 1) in one thread-block
// cluster.
//
// On the levels n <= 16 a V-cycle step (a residual, a smoothing sweep, a
// transfer) is a few microseconds of arithmetic, while a separate launch per
// step costs about 8-13 us of launch and ramp-up, and a grid-wide barrier
// through global atomics about 5-7 us.  This kernel runs MG(Kc, g, 0, m) for
// the levels n_Kc <= 16 .. n_0 in one launch of one cluster of CTAs, whose
// steps are separated by the hardware cluster barrier (release / acquire at
// cluster scope, which also orders the CTAs' global-memory writes):
//
//   pre-smoothing  z = S g ; m - 1 times { r = g - A z ; z += S r }
//   r = g - A z ; g_{k-1} = P^t r ; z_{k-1} = 0        (down to level 1)
//   z_0 = A_0^{-1} g_0                                  (coarsest)
//   z += P z_{k-1} ; m times { r = g - A z ; z += S r } (up to level Kc)
//
// with S = eta (sum_T J_T A_T^{-1} J_T^t + sum_V J_V W W^t J_V^t) of eq.
// (Preconditioner P) on CUDA cores in FP32 (one warp per vertex patch, W of
// every level in shared memory, overlapping patch outputs added with
// atomics), the operator as a direct 33-point stencil per edge in the
// factored form K = C^t M_F C, and the transfers of Sec. 3.1.
#include <cstring>

#include "coarse_cycle.cuh"

namespace ndmg {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kWStride = 61;                 // W rows padded to an odd stride (conflict-free both ways)
constexpr int kWarpScratch = 176;            // floats of per-warp scratch (gathered r_p, then W^t r_p)
constexpr int kMaxN0 = 108;                  // coarsest level 4^3 at most
constexpr int kCluster = 16;                 // CTAs of the cluster (one per SM)

struct Lv {
  int n;
  float cK, cM;        // alpha h / 6 and beta h^3 / 36 (integer stencil weights [1, 4, 1])
  float *g, *z, *r;
  const float* W;      // 108 x 60 Gram factor of the vertex-space operator
  const float* AinvT;  // 6 x 6 interior-space inverse
};

struct Args {
  int Kc, R, m, N0;
  float eta;
  Lv lv[kCoarseMaxLevels + 1];   // [0] coarsest (g, z only), [1 .. Kc]
  const double* Ainv0;           // N0 x N0 (symmetric)
  int* status;
};

// every thread of every CTA of the cluster: the step before is complete and
// its global-memory writes are visible to the whole cluster
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---- edges of level n (canonical layout of ndmg.h) ---------------------------
__host__ __device__ __forceinline__ int idx_x(int n, int i, int j, int k) {  // -1 when not interior
  return (unsigned)i < (unsigned)n && (unsigned)(j - 1) < (unsigned)(n - 1) && (unsigned)(k - 1) < (unsigned)(n - 1)
             ? ((k - 1) * (n - 1) + (j - 1)) * n + i
             : -1;
}
__host__ __device__ __forceinline__ int idx_y(int n, int i, int j, int k) {
  return (unsigned)(i - 1) < (unsigned)(n - 1) && (unsigned)j < (unsigned)n && (unsigned)(k - 1) < (unsigned)(n - 1)
             ? n * (n - 1) * (n - 1) + ((k - 1) * n + j) * (n - 1) + (i - 1)
             : -1;
}
__host__ __device__ __forceinline__ int idx_z(int n, int i, int j, int k) {
  return (unsigned)(i - 1) < (unsigned)(n - 1) && (unsigned)(j - 1) < (unsigned)(n - 1) && (unsigned)k < (unsigned)n
             ? 2 * n * (n - 1) * (n - 1) + (k * (n - 1) + (j - 1)) * (n - 1) + (i - 1)
             : -1;
}
__host__ __device__ __forceinline__ int idx_d(int n, int d, int i, int j, int k) {
  return d == 0 ? idx_x(n, i, j, k) : d == 1 ? idx_y(n, i, j, k) : idx_z(n, i, j, k);
}
__host__ __device__ __forceinline__ float at(const float* u, int e) { return e >= 0 ? u[e] : 0.f; }

// face circulations (face with lowest corner (i, j, k), normal x / y / z)
__host__ __device__ __forceinline__ float circ_x(const float* u, int n, int i, int j, int k) {
  return at(u, idx_z(n, i, j + 1, k)) - at(u, idx_z(n, i, j, k)) - at(u, idx_y(n, i, j, k + 1)) + at(u, idx_y(n, i, j, k));
}
__host__ __device__ __forceinline__ float circ_y(const float* u, int n, int i, int j, int k) {
  return at(u, idx_x(n, i, j, k + 1)) - at(u, idx_x(n, i, j, k)) - at(u, idx_z(n, i + 1, j, k)) + at(u, idx_z(n, i, j, k));
}
__host__ __device__ __forceinline__ float circ_z(const float* u, int n, int i, int j, int k) {
  return at(u, idx_y(n, i + 1, j, k)) - at(u, idx_y(n, i, j, k)) - at(u, idx_x(n, i, j + 1, k)) + at(u, idx_x(n, i, j, k));
}
// face masses along the normal, integer weights [1, 4, 1]
__host__ __device__ __forceinline__ float Xf(const float* u, int n, int i, int j, int k) {
  return circ_x(u, n, i - 1, j, k) + 4.f * circ_x(u, n, i, j, k) + circ_x(u, n, i + 1, j, k);
}
__host__ __device__ __forceinline__ float Yf(const float* u, int n, int i, int j, int k) {
  return circ_y(u, n, i, j - 1, k) + 4.f * circ_y(u, n, i, j, k) + circ_y(u, n, i, j + 1, k);
}
__host__ __device__ __forceinline__ float Zf(const float* u, int n, int i, int j, int k) {
  return circ_z(u, n, i, j, k - 1) + 4.f * circ_z(u, n, i, j, k) + circ_z(u, n, i, j, k + 1);
}

// (A u)_e for the edge of direction d at (i, j, k): cK (C^t M_F C u)_e + cM (M u)_e
__host__ __device__ float apply_edge(const Lv& L, const float* u, int d, int i, int j, int k) {
  const int n = L.n;
  float kv, mv = 0.f;
  const float w3[3] = {1.f, 4.f, 1.f};
  if (d == 0) {
    kv = (Yf(u, n, i, j, k - 1) - Yf(u, n, i, j, k)) + (Zf(u, n, i, j, k) - Zf(u, n, i, j - 1, k));
    for (int b = -1; b <= 1; ++b)
      for (int c = -1; c <= 1; ++c) mv += w3[b + 1] * w3[c + 1] * at(u, idx_x(n, i, j + b, k + c));
  } else if (d == 1) {
    kv = (Zf(u, n, i - 1, j, k) - Zf(u, n, i, j, k)) + (Xf(u, n, i, j, k) - Xf(u, n, i, j, k - 1));
    for (int a = -1; a <= 1; ++a)
      for (int c = -1; c <= 1; ++c) mv += w3[a + 1] * w3[c + 1] * at(u, idx_y(n, i + a, j, k + c));
  } else {
    kv = (Xf(u, n, i, j - 1, k) - Xf(u, n, i, j, k)) + (Yf(u, n, i, j, k) - Yf(u, n, i - 1, j, k));
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b) mv += w3[a + 1] * w3[b + 1] * at(u, idx_z(n, i + a, j + b, k));
  }
  return L.cK * kv + L.cM * mv;
}

// coordinates of edge e of level n
__host__ __device__ __forceinline__ void edge_coords(int n, int e, int* d, int* i, int* j, int* k) {
  const int n1 = n - 1, N3 = n * n1 * n1;
  *d = e / N3;
  int l = e - *d * N3;
  if (*d == 0) {
    *i = l % n; l /= n; *j = l % n1 + 1; *k = l / n1 + 1;
  } else if (*d == 1) {
    *i = l % n1 + 1; l /= n1; *j = l % n; *k = l / n + 1;
  } else {
    *i = l % n1 + 1; l /= n1; *j = l % n1 + 1; *k = l / n1;
  }
}

// edge of local index l (canonical numbering of the 4 x 4 x 4 box of cells)
// of vertex patch p (interior vertices, x fastest, nv per axis) on level n
__device__ __forceinline__ int patch_edge(int n, int nv, int p, int l) {
  const int vx = 1 + p % nv, vy = 1 + (p / nv) % nv, vz = 1 + p / (nv * nv);
  int d, bi, bj, bk;
  if (l < 36) {
    d = 0; bi = l % 4; bj = (l / 4) % 3 + 1; bk = l / 12 + 1;
  } else if (l < 72) {
    d = 1; bi = (l - 36) % 3 + 1; bj = ((l - 36) / 3) % 4; bk = (l - 36) / 12 + 1;
  } else {
    d = 2; bi = (l - 72) % 3 + 1; bj = ((l - 72) / 3) % 3 + 1; bk = (l - 72) / 9;
  }
  return idx_d(n, d, 2 * vx - 2 + bi, 2 * vy - 2 + bj, 2 * vz - 2 + bk);
}

// ---- phases ------------------------------------------------------------------
// r = g - A z (every right-hand side)
__device__ void phase_residual(const Lv& L, int R, int gtid, int gsize) {
  const int n = L.n, N = 3 * n * (n - 1) * (n - 1);
  for (int w = gtid; w < N * R; w += gsize) {
    const int rhs = w / N, e = w - rhs * N;
    int d, i, j, k;
    edge_coords(n, e, &d, &i, &j, &k);
    const float* z = L.z + (size_t)rhs * N;
    L.r[(size_t)rhs * N + e] = L.g[(size_t)rhs * N + e] - apply_edge(L, z, d, i, j, k);
  }
}

// z += eta * (interior solves + vertex-patch solves) of r (src); patch
// outputs overlap, so every contribution is an atomic add
__device__ void phase_smooth(const Args& A, const Lv& L, const float* src, const float* Wsm, float* wscr, int gtid,
                             int gsize, int gwarp, int nwarps, int lane) {
  const int n = L.n, nc = n / 2, nv = nc - 1, N = 3 * n * (n - 1) * (n - 1);
  // interior spaces: one thread per coarse element
  const int NT = nc * nc * nc;
  for (int w = gtid; w < NT * A.R; w += gsize) {
    const int rhs = w / NT, t = w - rhs * NT;
    const int I = t % nc, J = (t / nc) % nc, K = t / (nc * nc);
    const float* r = src + (size_t)rhs * N;
    float* z = L.z + (size_t)rhs * N;
    int g[6];
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        int p[3] = {2 * I + 1, 2 * J + 1, 2 * K + 1};
        p[d] = 2 * (d == 0 ? I : d == 1 ? J : K) + s;
        g[2 * d + s] = idx_d(n, d, p[0], p[1], p[2]);
      }
    float rv[6];
    for (int a = 0; a < 6; ++a) rv[a] = r[g[a]];
    for (int a = 0; a < 6; ++a) {
      float s = 0.f;
      for (int b = 0; b < 6; ++b) s += L.AinvT[a * 6 + b] * rv[b];
      atomicAdd(z + g[a], A.eta * s);
    }
  }
  // vertex patches: one warp per patch; local edge l of the patch of vertex
  // (vx, vy, vz) is edge (d, 2v - 2 + box coordinates) in the canonical order
  // of the 4 x 4 x 4 box of cells around it
  const int NP = nv * nv * nv;
  float* rp = wscr;        // 108 gathered values
  float* tp = wscr + 112;  // 60 coefficients W^t r_p
  for (int w = gwarp; w < NP * A.R; w += nwarps) {
    const int rhs = w / NP, p = w - rhs * NP;
    const int vx = 1 + p % nv, vy = 1 + (p / nv) % nv, vz = 1 + p / (nv * nv);
    const float* r = src + (size_t)rhs * N;
    float* z = L.z + (size_t)rhs * N;
    int gl[4];
    for (int q = 0; q < 4; ++q) {
      const int l = lane + 32 * q;
      gl[q] = -1;
      if (l < 108) {
        int d, bi, bj, bk;
        if (l < 36) {
          d = 0; bi = l % 4; bj = (l / 4) % 3 + 1; bk = l / 12 + 1;
        } else if (l < 72) {
          d = 1; bi = (l - 36) % 3 + 1; bj = ((l - 36) / 3) % 4; bk = (l - 36) / 12 + 1;
        } else {
          d = 2; bi = (l - 72) % 3 + 1; bj = ((l - 72) / 3) % 3 + 1; bk = (l - 72) / 9;
        }
        gl[q] = idx_d(n, d, 2 * vx - 2 + bi, 2 * vy - 2 + bj, 2 * vz - 2 + bk);
        rp[l] = gl[q] >= 0 ? r[gl[q]] : 0.f;
      }
    }
    __syncwarp();
    for (int c = lane; c < 60; c += 32) {
      float s = 0.f;
      for (int l = 0; l < 108; ++l) s += Wsm[l * kWStride + c] * rp[l];
      tp[c] = s;
    }
    __syncwarp();
    for (int q = 0; q < 4; ++q) {
      const int l = lane + 32 * q;
      if (l < 108 && gl[q] >= 0) {
        float s = 0.f;
        for (int c = 0; c < 60; ++c) s += Wsm[l * kWStride + c] * tp[c];
        atomicAdd(z + gl[q], A.eta * s);
      }
    }
    __syncwarp();
  }
}

// g_c = P^t r_f (coarse lattice point: its x-, y-, z-edge) and z_c = 0
__device__ void phase_restrict(const Lv& F, const Lv& C, int R, int gtid, int gsize) {
  const int nf = F.n, nc = C.n, Nf = 3 * nf * (nf - 1) * (nf - 1), Nc = 3 * nc * (nc - 1) * (nc - 1);
  const int NL = nc * nc * nc;
  const float w[3] = {0.5f, 1.f, 0.5f};
  for (int t = gtid; t < NL * R; t += gsize) {
    const int rhs = t / NL, q = t - rhs * NL;
    const int I = q % nc, J = (q / nc) % nc, K = q / (nc * nc);
    const float* rf = F.r + (size_t)rhs * Nf;
    float* gc = C.g + (size_t)rhs * Nc;
    float* zc = C.z + (size_t)rhs * Nc;
    int e = idx_x(nc, I, J, K);
    if (e >= 0) {
      float s = 0.f;
      for (int c = -1; c <= 1; ++c)
        for (int b = -1; b <= 1; ++b)
          for (int a = 0; a < 2; ++a) s += w[b + 1] * w[c + 1] * at(rf, idx_x(nf, 2 * I + a, 2 * J + b, 2 * K + c));
      gc[e] = s;
      zc[e] = 0.f;
    }
    e = idx_y(nc, I, J, K);
    if (e >= 0) {
      float s = 0.f;
      for (int c = -1; c <= 1; ++c)
        for (int a = 0; a < 2; ++a)
          for (int b = -1; b <= 1; ++b) s += w[b + 1] * w[c + 1] * at(rf, idx_y(nf, 2 * I + b, 2 * J + a, 2 * K + c));
      gc[e] = s;
      zc[e] = 0.f;
    }
    e = idx_z(nc, I, J, K);
    if (e >= 0) {
      float s = 0.f;
      for (int a = 0; a < 2; ++a)
        for (int c = -1; c <= 1; ++c)
          for (int b = -1; b <= 1; ++b) s += w[b + 1] * w[c + 1] * at(rf, idx_z(nf, 2 * I + b, 2 * J + c, 2 * K + a));
      gc[e] = s;
      zc[e] = 0.f;
    }
  }
}

// z_f += P z_c: one thread per coarse cell updates the 24 fine edges whose
// lowest node is in its 2 x 2 x 2 block (each fine edge has exactly one such cell)
__device__ void phase_prolong(const Lv& F, const Lv& C, int R, int gtid, int gsize) {
  const int nf = F.n, nc = C.n, Nf = 3 * nf * (nf - 1) * (nf - 1), Nc = 3 * nc * (nc - 1) * (nc - 1);
  const int NCELL = nc * nc * nc;
  for (int t = gtid; t < NCELL * R; t += gsize) {
    const int rhs = t / NCELL, q = t - rhs * NCELL;
    const int I = q % nc, J = (q / nc) % nc, K = q / (nc * nc);
    const float* zc = C.z + (size_t)rhs * Nc;
    float* zf = F.z + (size_t)rhs * Nf;
    float X[2][2], Y[2][2], Z[2][2];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        X[a][b] = at(zc, idx_x(nc, I, J + a, K + b));
        Y[a][b] = at(zc, idx_y(nc, I + a, J, K + b));
        Z[a][b] = at(zc, idx_z(nc, I + a, J + b, K));
      }
    auto lerp = [](const float (&V)[2][2], int d1, int d2) {
      const float v0 = d1 ? 0.5f * (V[0][0] + V[1][0]) : V[0][0];
      const float v1 = d1 ? 0.5f * (V[0][1] + V[1][1]) : V[0][1];
      return d2 ? 0.5f * (v0 + v1) : v0;
    };
    for (int d2 = 0; d2 < 2; ++d2)
      for (int d1 = 0; d1 < 2; ++d1)
        for (int s = 0; s < 2; ++s) {
          int e = idx_x(nf, 2 * I + s, 2 * J + d1, 2 * K + d2);
          if (e >= 0) zf[e] += lerp(X, d1, d2);
          e = idx_y(nf, 2 * I + d1, 2 * J + s, 2 * K + d2);
          if (e >= 0) zf[e] += lerp(Y, d1, d2);
          e = idx_z(nf, 2 * I + d1, 2 * J + d2, 2 * K + s);
          if (e >= 0) zf[e] += lerp(Z, d1, d2);
        }
  }
}

// z_0 = A_0^{-1} g_0: one warp per row (the inverse is symmetric)
__device__ void phase_coarse(const Args& A, int gwarp, int nwarps, int lane) {
  const int N0 = A.N0;
  for (int w = gwarp; w < N0 * A.R; w += nwarps) {
    const int rhs = w / N0, row = w - rhs * N0;
    const float* g = A.lv[0].g + (size_t)rhs * N0;
    double s = 0.0;
    for (int j = lane; j < N0; j += 32) s += A.Ainv0[(size_t)row * N0 + j] * (double)g[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) A.lv[0].z[(size_t)rhs * N0 + row] = (float)s;
  }
}

__global__ void __launch_bounds__(kThreads) k_coarse_vcycle(Args A) {
  extern __shared__ __align__(16) float sm[];
  if (*reinterpret_cast<volatile int*>(A.status) != 0) return;
  float* Wall = sm;                                     // Kc levels x 108 x kWStride
  float* wscr = sm + A.Kc * 108 * kWStride + (threadIdx.x >> 5) * kWarpScratch;
  for (int k = 1; k <= A.Kc; ++k)
    for (int q = threadIdx.x; q < 108 * 60; q += kThreads)
      Wall[(k - 1) * 108 * kWStride + (q / 60) * kWStride + q % 60] = A.lv[k].W[q];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int gtid = blockIdx.x * kThreads + threadIdx.x, gsize = gridDim.x * kThreads;
  const int gwarp = blockIdx.x * kWarps + (threadIdx.x >> 5), nwarps = gridDim.x * kWarps;
  auto Wof = [&](int k) { return Wall + (k - 1) * 108 * kWStride; };
#define NDMG_BARRIER() cluster_sync()
  // down: level Kc .. 1 (z_Kc = 0 on entry, coarser z zeroed by the restriction)
  for (int k = A.Kc; k >= 1; --k) {
    const Lv& L = A.lv[k];
    phase_smooth(A, L, L.g, Wof(k), wscr, gtid, gsize, gwarp, nwarps, lane);   // z = S g (z = 0)
    NDMG_BARRIER();
    for (int s = 1; s < A.m; ++s) {
      phase_residual(L, A.R, gtid, gsize);
      NDMG_BARRIER();
      phase_smooth(A, L, L.r, Wof(k), wscr, gtid, gsize, gwarp, nwarps, lane);
      NDMG_BARRIER();
    }
    phase_residual(L, A.R, gtid, gsize);
    NDMG_BARRIER();
    phase_restrict(L, A.lv[k - 1], A.R, gtid, gsize);
    NDMG_BARRIER();
  }
  phase_coarse(A, gwarp, nwarps, lane);
  NDMG_BARRIER();
  // up: level 1 .. Kc
  for (int k = 1; k <= A.Kc; ++k) {
    const Lv& L = A.lv[k];
    phase_prolong(L, A.lv[k - 1], A.R, gtid, gsize);
    NDMG_BARRIER();
    for (int s = 0; s < A.m; ++s) {
      phase_residual(L, A.R, gtid, gsize);
      NDMG_BARRIER();
      phase_smooth(A, L, L.r, Wof(k), wscr, gtid, gsize, gwarp, nwarps, lane);
      if (k < A.Kc || s + 1 < A.m) NDMG_BARRIER();
    }
  }
#undef NDMG_BARRIER
}

size_t coarse_smem(int Kc) {
  // W of every level, then the per-warp scratch (16-byte aligned: 108 * 61 * 4 * Kc is a multiple of 16)
  return sizeof(float) * ((size_t)Kc * 108 * kWStride + (size_t)kWarps * kWarpScratch);
}

}  // namespace

cudaError_t prepare_coarse_cycle() {
  cudaError_t e = cudaFuncSetAttribute(k_coarse_vcycle, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)coarse_smem(kCoarseMaxLevels));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_coarse_vcycle, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

static cudaLaunchConfig_t cluster_config(int Kc, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCluster);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = coarse_smem(Kc);
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

int coarse_cycle_grid(int, int Kc) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config(Kc, nullptr, attr);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_coarse_vcycle, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return 0;
  }
  return kCluster;
}

cudaError_t launch_coarse_cycle(cudaStream_t s, int grid, const CoarseLevel* lv, int Kc, int N0, const double* Ainv0,
                                float* g0, float* z0, double eta, int m, int R, int* status) {
  if (Kc < 1 || Kc > kCoarseMaxLevels || N0 > kMaxN0 || grid != kCluster) return cudaErrorInvalidValue;
  Args a;
  std::memset(&a, 0, sizeof(a));
  a.Kc = Kc;
  a.R = R;
  a.m = m;
  a.N0 = N0;
  a.eta = (float)eta;
  a.lv[0].g = g0;
  a.lv[0].z = z0;
  for (int k = 1; k <= Kc; ++k) {
    const CoarseLevel& c = lv[k];
    a.lv[k].n = c.n;
    a.lv[k].cK = (float)(c.cK / 6.0);
    a.lv[k].cM = (float)(c.cM / 36.0);
    a.lv[k].g = c.g;
    a.lv[k].z = c.z;
    a.lv[k].r = c.r;
    a.lv[k].W = c.W;
    a.lv[k].AinvT = c.AinvT;
  }
  a.lv[0].n = lv[0].n;
  a.Ainv0 = Ainv0;
  a.status = status;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config(Kc, s, attr);
  return cudaLaunchKernelEx(&cfg, k_coarse_vcycle, a);
}

}  // namespace ndmg
