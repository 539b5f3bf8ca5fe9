// CUDA-core kernels of the V-cycle: matrix-free operator apply / residual,
// grid transfers, interior-space and vertex-patch smoother pieces, coarsest
// solve and FP64 reductions.  Templated on the vector element type
// (double for the FP64 path, float for the mixed path's inner V-cycle).
#include "kernels.cuh"

namespace ndmg {

// ---------------------------------------------------------------------------
// Edge lattice helpers (layout of ndmg.h): per-direction offsets.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t off_x(int n, int i, int j, int k) {
  return ((int64_t)(k - 1) * (n - 1) + (j - 1)) * n + i;
}
__device__ __forceinline__ int64_t off_y(int n, int i, int j, int k) {
  return ((int64_t)(k - 1) * n + j) * (n - 1) + (i - 1);
}
__device__ __forceinline__ int64_t off_z(int n, int i, int j, int k) {
  return ((int64_t)k * (n - 1) + (j - 1)) * (n - 1) + (i - 1);
}
__device__ __forceinline__ bool in_seg(int p, int n) { return (unsigned)p < (unsigned)n; }
__device__ __forceinline__ bool in_node(int p, int n) { return (unsigned)(p - 1) < (unsigned)(n - 1); }

// value of an edge, zero on the boundary and outside the box
template <typename T>
__device__ __forceinline__ T UX(const T* __restrict__ u, int n, int i, int j, int k) {
  return (in_seg(i, n) && in_node(j, n) && in_node(k, n)) ? __ldg(u + off_x(n, i, j, k)) : T(0);
}
template <typename T>
__device__ __forceinline__ T UY(const T* __restrict__ u, int n, int i, int j, int k) {
  return (in_node(i, n) && in_seg(j, n) && in_node(k, n)) ? __ldg(u + off_y(n, i, j, k)) : T(0);
}
template <typename T>
__device__ __forceinline__ T UZ(const T* __restrict__ u, int n, int i, int j, int k) {
  return (in_node(i, n) && in_node(j, n) && in_seg(k, n)) ? __ldg(u + off_z(n, i, j, k)) : T(0);
}

// decode a per-direction offset into lattice coordinates
__device__ __forceinline__ void decode(int d, int n, int64_t loc, int& i, int& j, int& k) {
  const int n1 = n - 1;
  if (d == 0) {
    i = (int)(loc % n);
    int64_t t = loc / n;
    j = (int)(t % n1) + 1;
    k = (int)(t / n1) + 1;
  } else if (d == 1) {
    i = (int)(loc % n1) + 1;
    int64_t t = loc / n1;
    j = (int)(t % n);
    k = (int)(t / n) + 1;
  } else {
    i = (int)(loc % n1) + 1;
    int64_t t = loc / n1;
    j = (int)(t % n1) + 1;
    k = (int)(t / n1);
  }
}

// ---------------------------------------------------------------------------
// Operator apply.  A = alpha K + beta M with K = h C^t Mf C: C is the integer
// edge->face circulation matrix, Mf the face mass along the face normal
// ([1/6, 2/3, 1/6], zero on boundary planes); M is the edge mass, a 3x3
// tensor stencil [1/6,2/3,1/6]^2 across the edge.  cK = alpha h, cM = beta h^3.
// Face circulations (normal x, y, z) of the face whose lowest corner is the
// node/segment triple (i, j, k):
//   cx(i,j,k) = uz(i,j+1,k) - uz(i,j,k) - uy(i,j,k+1) + uy(i,j,k)
//   cy(i,j,k) = ux(i,j,k+1) - ux(i,j,k) - uz(i+1,j,k) + uz(i,j,k)
//   cz(i,j,k) = uy(i+1,j,k) - uy(i,j,k) - ux(i,j+1,k) + ux(i,j,k)
// ---------------------------------------------------------------------------
template <typename T>
struct Fields {
  const T* __restrict__ ux;
  const T* __restrict__ uy;
  const T* __restrict__ uz;
  int n;
  __device__ __forceinline__ T cx(int i, int j, int k) const {
    return UZ(uz, n, i, j + 1, k) - UZ(uz, n, i, j, k) - UY(uy, n, i, j, k + 1) + UY(uy, n, i, j, k);
  }
  __device__ __forceinline__ T cy(int i, int j, int k) const {
    return UX(ux, n, i, j, k + 1) - UX(ux, n, i, j, k) - UZ(uz, n, i + 1, j, k) + UZ(uz, n, i, j, k);
  }
  __device__ __forceinline__ T cz(int i, int j, int k) const {
    return UY(uy, n, i + 1, j, k) - UY(uy, n, i, j, k) - UX(ux, n, i, j + 1, k) + UX(ux, n, i, j, k);
  }
  // face mass along the normal
  __device__ __forceinline__ T Xf(int i, int j, int k) const {
    return T(1.0 / 6.0) * (cx(i - 1, j, k) + cx(i + 1, j, k)) + T(2.0 / 3.0) * cx(i, j, k);
  }
  __device__ __forceinline__ T Yf(int i, int j, int k) const {
    return T(1.0 / 6.0) * (cy(i, j - 1, k) + cy(i, j + 1, k)) + T(2.0 / 3.0) * cy(i, j, k);
  }
  __device__ __forceinline__ T Zf(int i, int j, int k) const {
    return T(1.0 / 6.0) * (cz(i, j, k - 1) + cz(i, j, k + 1)) + T(2.0 / 3.0) * cz(i, j, k);
  }
};

template <typename T>
__device__ __forceinline__ T mass3x3(T m1, T c, T p1) {
  return T(1.0 / 6.0) * (m1 + p1) + T(2.0 / 3.0) * c;
}

template <typename T>
__device__ __forceinline__ T apply_edge(const Fields<T>& F, int d, int i, int j, int k, T cK, T cM) {
  const int n = F.n;
  T kv, mv;
  if (d == 0) {
    kv = -F.Yf(i, j, k) + F.Yf(i, j, k - 1) + F.Zf(i, j, k) - F.Zf(i, j - 1, k);
    T r[3];
#pragma unroll
    for (int b = -1; b <= 1; ++b)
      r[b + 1] = mass3x3(UX(F.ux, n, i, j - 1, k + b), UX(F.ux, n, i, j, k + b), UX(F.ux, n, i, j + 1, k + b));
    mv = mass3x3(r[0], r[1], r[2]);
  } else if (d == 1) {
    kv = -F.Zf(i, j, k) + F.Zf(i - 1, j, k) + F.Xf(i, j, k) - F.Xf(i, j, k - 1);
    T r[3];
#pragma unroll
    for (int b = -1; b <= 1; ++b)
      r[b + 1] = mass3x3(UY(F.uy, n, i - 1, j, k + b), UY(F.uy, n, i, j, k + b), UY(F.uy, n, i + 1, j, k + b));
    mv = mass3x3(r[0], r[1], r[2]);
  } else {
    kv = -F.Xf(i, j, k) + F.Xf(i, j - 1, k) + F.Yf(i, j, k) - F.Yf(i - 1, j, k);
    T r[3];
#pragma unroll
    for (int b = -1; b <= 1; ++b)
      r[b + 1] = mass3x3(UZ(F.uz, n, i - 1, j + b, k), UZ(F.uz, n, i, j + b, k), UZ(F.uz, n, i + 1, j + b, k));
    mv = mass3x3(r[0], r[1], r[2]);
  }
  return cK * kv + cM * mv;
}

// y = A u (g == nullptr) or y = g - A u
template <typename T>
__global__ void __launch_bounds__(256) k_stencil(int n, T cK, T cM, const T* __restrict__ u,
                                                 const T* __restrict__ g, T* __restrict__ y) {
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  Fields<T> F{u, u + N3, u + 2 * N3, n};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * N3;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(e / N3);
    int i, j, k;
    decode(d, n, e - d * N3, i, j, k);
    const T v = apply_edge(F, d, i, j, k, cK, cM);
    y[e] = g ? g[e] - v : v;
  }
}

// ---------------------------------------------------------------------------
// Grid transfer (Sec. 3.1).  Prolongation = natural injection N_{k-1} ->
// N_k: along a coarse edge both fine halves take its value; across it the
// coarse hat is linear (weight 1 at the coarse node, 1/2 one fine node away).
// Restriction is the transpose.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(int nf, const T* __restrict__ rf, T* __restrict__ gc) {
  const int nc = nf / 2;
  const int64_t N3c = (int64_t)nc * (nc - 1) * (nc - 1);
  const int64_t N3f = (int64_t)nf * (nf - 1) * (nf - 1);
  const T w[3] = {T(0.5), T(1), T(0.5)};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * N3c;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(e / N3c);
    int I, J, K;
    decode(d, nc, e - d * N3c, I, J, K);
    const T* r = rf + d * N3f;
    T s = T(0);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = -1; b <= 1; ++b)
#pragma unroll
        for (int c = -1; c <= 1; ++c) {
          const T wt = w[b + 1] * w[c + 1];
          if (d == 0) s += wt * __ldg(r + off_x(nf, 2 * I + a, 2 * J + b, 2 * K + c));
          else if (d == 1) s += wt * __ldg(r + off_y(nf, 2 * I + c, 2 * J + a, 2 * K + b));
          else s += wt * __ldg(r + off_z(nf, 2 * I + b, 2 * J + c, 2 * K + a));
        }
    gc[e] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(int nf, const T* __restrict__ zc, T* __restrict__ zf) {
  const int nc = nf / 2;
  const int64_t N3c = (int64_t)nc * (nc - 1) * (nc - 1);
  const int64_t N3f = (int64_t)nf * (nf - 1) * (nf - 1);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * N3f;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(e / N3f);
    int p[3];
    decode(d, nf, e - d * N3f, p[0], p[1], p[2]);
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    int c[3];
    c[d] = p[d] >> 1;
    // transverse coarse nodes and weights
    int na = (p[t1] & 1) ? 2 : 1, nb = (p[t2] & 1) ? 2 : 1;
    int A[2] = {p[t1] >> 1, (p[t1] >> 1) + 1}, B[2] = {p[t2] >> 1, (p[t2] >> 1) + 1};
    const T wa = (na == 2) ? T(0.5) : T(1), wb = (nb == 2) ? T(0.5) : T(1);
    const T* z = zc + d * N3c;
    T s = T(0);
    for (int a = 0; a < na; ++a)
      for (int b = 0; b < nb; ++b) {
        c[t1] = A[a];
        c[t2] = B[b];
        if (!in_node(c[t1], nc) || !in_node(c[t2], nc)) continue;
        int64_t o = d == 0 ? off_x(nc, c[0], c[1], c[2]) : d == 1 ? off_y(nc, c[0], c[1], c[2]) : off_z(nc, c[0], c[1], c[2]);
        s += wa * wb * __ldg(z + o);
      }
    zf[e] += s;
  }
}

// ---------------------------------------------------------------------------
// Smoother, eq. (Preconditioner P): z += eta (sum_T J_T A_T^{-1} J_T^t r +
// sum_V J_V A_V^{-1} J_V^t r).  Interior spaces (eq. SubdomainSpace): the 6
// fine edges strictly inside each coarse element, disjoint, so each thread
// owns its 6 outputs.  Local order = the 2x2x2 box numbering (x, y, z edges,
// segment 0 then 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t edge_gidx(int n, int d, int i, int j, int k) {
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  return d == 0 ? off_x(n, i, j, k) : d == 1 ? N3 + off_y(n, i, j, k) : 2 * N3 + off_z(n, i, j, k);
}

template <typename T>
__global__ void __launch_bounds__(256) k_bubble(int n, const T* __restrict__ Ainv, T eta, const T* __restrict__ r,
                                                T* __restrict__ z) {
  const int nc = n / 2;
  const int64_t NT = (int64_t)nc * nc * nc;
  __shared__ T As[36];
  if (threadIdx.x < 36) As[threadIdx.x] = Ainv[threadIdx.x];
  __syncthreads();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < NT; t += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(t % nc), J = (int)((t / nc) % nc), K = (int)(t / ((int64_t)nc * nc));
    int64_t g[6];
    int q = 0;
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        int p[3] = {2 * I + 1, 2 * J + 1, 2 * K + 1};
        p[d] = (d == 0 ? 2 * I : d == 1 ? 2 * J : 2 * K) + s;
        g[q++] = edge_gidx(n, d, p[0], p[1], p[2]);
      }
    T rv[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) rv[a] = __ldg(r + g[a]);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      T s = T(0);
#pragma unroll
      for (int b = 0; b < 6; ++b) s += As[a * 6 + b] * rv[b];
      z[g[a]] += eta * s;
    }
  }
}

// Vertex patch local index l in [0,108) -> global edge, patch at coarse
// vertex (I,J,K): the 4x4x4 box numbering with origin (2I-2, 2J-2, 2K-2).
__device__ __forceinline__ int64_t patch_gidx(int n, int I, int J, int K, int l) {
  int d, i, j, k;
  if (l < 36) {
    d = 0; i = l % 4; j = (l / 4) % 3 + 1; k = l / 12 + 1;
  } else if (l < 72) {
    l -= 36; d = 1; i = l % 3 + 1; j = (l / 3) % 4; k = l / 12 + 1;
  } else {
    l -= 72; d = 2; i = l % 3 + 1; j = (l / 3) % 3 + 1; k = l / 9;
  }
  return edge_gidx(n, d, 2 * I - 2 + i, 2 * J - 2 + j, 2 * K - 2 + k);
}

// Dense vertex-patch solve on CUDA cores: z += eta * D r_p per patch, D =
// J_V A_V^{-1} J_V^t (108x108, symmetric) staged in shared memory, PB patches
// per pass; overlapping patches accumulate with atomics.
template <typename T, int PB>
__global__ void __launch_bounds__(128) k_vertex_dense(int n, const T* __restrict__ D, T eta, const T* __restrict__ r,
                                                      T* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ds = reinterpret_cast<T*>(smem_raw);          // 108*108
  T* Rs = Ds + 108 * 108;                          // 108*PB
  const int nc = n / 2, nv = nc - 1;
  const int64_t NP = (int64_t)nv * nv * nv;
  for (int q = threadIdx.x; q < 108 * 108; q += blockDim.x) Ds[q] = D[q];
  for (int64_t base = (int64_t)blockIdx.x * PB; base < NP; base += (int64_t)gridDim.x * PB) {
    __syncthreads();
    for (int q = threadIdx.x; q < 108 * PB; q += blockDim.x) {
      const int p = q / 108, l = q % 108;
      const int64_t P = base + p;
      T v = T(0);
      if (P < NP) {
        const int I = (int)(P % nv) + 1, J = (int)((P / nv) % nv) + 1, K = (int)(P / ((int64_t)nv * nv)) + 1;
        v = __ldg(r + patch_gidx(n, I, J, K, l));
      }
      Rs[l * PB + p] = v;
    }
    __syncthreads();
    for (int row = threadIdx.x; row < 108; row += blockDim.x) {
      T acc[PB];
#pragma unroll
      for (int p = 0; p < PB; ++p) acc[p] = T(0);
      for (int c = 0; c < 108; ++c) {
        const T dv = Ds[c * 108 + row];
#pragma unroll
        for (int p = 0; p < PB; ++p) acc[p] += dv * Rs[c * PB + p];
      }
#pragma unroll
      for (int p = 0; p < PB; ++p) {
        const int64_t P = base + p;
        if (P < NP) {
          const int I = (int)(P % nv) + 1, J = (int)((P / nv) % nv) + 1, K = (int)(P / ((int64_t)nv * nv)) + 1;
          atomicAdd(z + patch_gidx(n, I, J, K, row), eta * acc[p]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Coarsest solve (Fig. 1, k = 0): z = A_0^{-1} g with the precomputed dense
// inverse, one CTA.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_coarse(int N0, const double* __restrict__ Ainv, const T* __restrict__ g,
                                                T* __restrict__ z) {
  extern __shared__ double gs[];
  for (int i = threadIdx.x; i < N0; i += blockDim.x) gs[i] = (double)g[i];
  __syncthreads();
  for (int i = threadIdx.x; i < N0; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < N0; ++j) s += Ainv[(int64_t)j * N0 + i] * gs[j];
    z[i] = (T)s;
  }
}

// ---------------------------------------------------------------------------
// BLAS-1 with FP64 accumulation.  Reductions are two-stage and deterministic:
// a fixed number of blocks writes partial sums, one block adds them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* out) {
  __shared__ double ws[NV][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = warp_sum(v[a]);
  if (lane == 0)
#pragma unroll
    for (int a = 0; a < NV; ++a) ws[a][w] = v[a];
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double s = lane < nw ? ws[a][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) out[a] = s;
    }
  }
}

// partial[b*2 + {0,1}] = block sums of x.y and (optionally) x2.y2
template <typename T>
__global__ void __launch_bounds__(256) k_dot2(int64_t N, const T* __restrict__ x, const T* __restrict__ y,
                                              const T* __restrict__ x2, const T* __restrict__ y2,
                                              double* __restrict__ partial) {
  double v[2] = {0.0, 0.0};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    v[0] += (double)x[e] * (double)y[e];
    if (x2) v[1] += (double)x2[e] * (double)y2[e];
  }
  block_sum_store<2>(v, partial + 2 * blockIdx.x);
}

__global__ void k_finish2(int nb, const double* __restrict__ partial, double* __restrict__ out) {
  double v[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    v[0] += partial[2 * b];
    v[1] += partial[2 * b + 1];
  }
  block_sum_store<2>(v, out);
}

// y = a x + b y
template <typename T>
__global__ void __launch_bounds__(256) k_axpby(int64_t N, double a, const T* __restrict__ x, double b, T* __restrict__ y) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (T)(a * (double)x[e] + b * (double)y[e]);
}

// u += a p ; r -= a q
template <typename T>
__global__ void __launch_bounds__(256) k_cg_update(int64_t N, double a, const T* __restrict__ p, const T* __restrict__ q,
                                                   T* __restrict__ u, T* __restrict__ r) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    u[e] = (T)((double)u[e] + a * (double)p[e]);
    r[e] = (T)((double)r[e] - a * (double)q[e]);
  }
}

// dst (float) = s * src (double)
__global__ void __launch_bounds__(256) k_to_f32(int64_t N, double s, const double* __restrict__ src, float* __restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (float)(s * src[e]);
}

// dst (double) += s * src (float)
__global__ void __launch_bounds__(256) k_add_f32(int64_t N, double s, const float* __restrict__ src, double* __restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] += s * (double)src[e];
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static inline int grid_for(int64_t work, int sm_count, int per_sm = 8) {
  int64_t b = (work + 255) / 256;
  int64_t cap = (int64_t)sm_count * per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T>
void launch_stencil(cudaStream_t s, int sm, int n, double cK, double cM, const T* u, const T* g, T* y) {
  const int64_t N = 3LL * n * (n - 1) * (n - 1);
  if (N == 0) return;
  k_stencil<T><<<grid_for(N, sm, 16), 256, 0, s>>>(n, (T)cK, (T)cM, u, g, y);
}

template <typename T>
void launch_restrict(cudaStream_t s, int sm, int nf, const T* rf, T* gc) {
  const int nc = nf / 2;
  const int64_t N = 3LL * nc * (nc - 1) * (nc - 1);
  if (N == 0) return;
  k_restrict<T><<<grid_for(N, sm, 16), 256, 0, s>>>(nf, rf, gc);
}

template <typename T>
void launch_prolong_add(cudaStream_t s, int sm, int nf, const T* zc, T* zf) {
  const int64_t N = 3LL * nf * (nf - 1) * (nf - 1);
  k_prolong_add<T><<<grid_for(N, sm, 16), 256, 0, s>>>(nf, zc, zf);
}

template <typename T>
void launch_bubble(cudaStream_t s, int sm, int n, const T* Ainv, double eta, const T* r, T* z) {
  const int64_t nc = n / 2;
  k_bubble<T><<<grid_for(nc * nc * nc, sm, 16), 256, 0, s>>>(n, Ainv, (T)eta, r, z);
}

constexpr int kPB64 = 8;
constexpr int kPB32 = 16;

template <typename T>
static constexpr int pb_for() { return sizeof(T) == 8 ? kPB64 : kPB32; }

template <typename T>
size_t vertex_dense_smem() { return sizeof(T) * (108 * 108 + 108 * pb_for<T>()); }

template <typename T>
cudaError_t prepare_vertex_dense() {
  return cudaFuncSetAttribute(k_vertex_dense<T, pb_for<T>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)vertex_dense_smem<T>());
}

template <typename T>
void launch_vertex_dense(cudaStream_t s, int sm, int n, const T* D, double eta, const T* r, T* z) {
  const int64_t nv = n / 2 - 1;
  const int64_t NP = nv * nv * nv;
  if (NP <= 0) return;
  constexpr int PB = pb_for<T>();
  int64_t blocks = (NP + PB - 1) / PB;
  const int64_t cap = (int64_t)sm * 2;
  if (blocks > cap) blocks = cap;
  k_vertex_dense<T, PB><<<(int)blocks, 128, vertex_dense_smem<T>(), s>>>(n, D, (T)eta, r, z);
}

template <typename T>
void launch_coarse(cudaStream_t s, int N0, const double* Ainv, const T* g, T* z) {
  k_coarse<T><<<1, 256, sizeof(double) * N0, s>>>(N0, Ainv, g, z);
}

int reduction_blocks(int sm) { return sm * 4; }

template <typename T>
void launch_dot2(cudaStream_t s, int sm, int64_t N, const T* x, const T* y, const T* x2, const T* y2, double* partial,
                 double* out) {
  const int nb = reduction_blocks(sm);
  k_dot2<T><<<nb, 256, 0, s>>>(N, x, y, x2, y2, partial);
  k_finish2<<<1, 256, 0, s>>>(nb, partial, out);
}

template <typename T>
void launch_axpby(cudaStream_t s, int sm, int64_t N, double a, const T* x, double b, T* y) {
  k_axpby<T><<<grid_for(N, sm, 8), 256, 0, s>>>(N, a, x, b, y);
}

template <typename T>
void launch_cg_update(cudaStream_t s, int sm, int64_t N, double a, const T* p, const T* q, T* u, T* r) {
  k_cg_update<T><<<grid_for(N, sm, 8), 256, 0, s>>>(N, a, p, q, u, r);
}

void launch_to_f32(cudaStream_t s, int sm, int64_t N, double sc, const double* src, float* dst) {
  k_to_f32<<<grid_for(N, sm, 8), 256, 0, s>>>(N, sc, src, dst);
}
void launch_add_f32(cudaStream_t s, int sm, int64_t N, double sc, const float* src, double* dst) {
  k_add_f32<<<grid_for(N, sm, 8), 256, 0, s>>>(N, sc, src, dst);
}

#define NDMG_INST(T)                                                                                   \
  template void launch_stencil<T>(cudaStream_t, int, int, double, double, const T*, const T*, T*);    \
  template void launch_restrict<T>(cudaStream_t, int, int, const T*, T*);                             \
  template void launch_prolong_add<T>(cudaStream_t, int, int, const T*, T*);                          \
  template void launch_bubble<T>(cudaStream_t, int, int, const T*, double, const T*, T*);             \
  template cudaError_t prepare_vertex_dense<T>();                                                     \
  template void launch_vertex_dense<T>(cudaStream_t, int, int, const T*, double, const T*, T*);       \
  template void launch_coarse<T>(cudaStream_t, int, const double*, const T*, T*);                     \
  template void launch_dot2<T>(cudaStream_t, int, int64_t, const T*, const T*, const T*, const T*,    \
                               double*, double*);                                                     \
  template void launch_axpby<T>(cudaStream_t, int, int64_t, double, const T*, double, T*);            \
  template void launch_cg_update<T>(cudaStream_t, int, int64_t, double, const T*, const T*, T*, T*);
NDMG_INST(double)
NDMG_INST(float)

}  // namespace ndmg
