// CUDA-core kernels of the V-cycle: matrix-free operator apply / residual,
// grid transfers, interior-space and vertex-patch smoother pieces, coarsest
// solve and FP64 reductions.  Templated on the vector element type
// (double for the FP64 path, float for the mixed path's inner V-cycle).
#include <type_traits>

#include "fpbits.cuh"
#include "kernels.cuh"
#include "pdl.cuh"

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
// Streaming variant: one CTA owns a column of TX x TY cells and walks a chunk
// of KZ planes along z (the edges whose lowest node is in the column).  Per
// plane it needs u on that plane and the next one (tile plus a one-cell halo
// in x and y), so u sits in a ring of three shared-memory planes and the next
// plane is staged with asynchronous copies (zero fill outside the box, which
// is exactly the boundary condition) while the current one is consumed; g is
// staged one plane ahead as well.  The three face-circulation planes are
// formed once per step in shared memory; the face mass along z and the edge
// mass across x- and y-edges, which span three planes, are carried in
// registers from one plane to the next.
constexpr int kTX = 32, kTY = 8;
constexpr int kPX = kTX + 2, kPY = kTY + 2, kP = kPX * kPY;  // one staged plane
constexpr int kTP = kTX * kTY;                               // outputs per plane
static_assert(kTX == 32, "one warp per row of a stencil block");

// asynchronous copy of one element global -> shared; zero fill when !valid
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid, const T* any_valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const void* sp = valid ? (const void*)src : (const void*)any_valid;
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(sp), "r"(valid ? 8u : 0u) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(sp), "r"(valid ? 4u : 0u) : "memory");
}

// In-plane part of one staged position (a, b) of the tile's plane: global
// offsets (without the plane term) and whether the x-, y-, z-edge there is
// interior as far as i and j decide; fixed for the whole column.
struct PlanePos {
  uint32_t ox, oy, oz;
  bool vx, vy, vz;
};

__device__ __forceinline__ PlanePos plane_pos(int n, int i, int j) {
  const uint32_t n1 = n - 1;
  PlanePos p;
  p.vx = in_seg(i, n) && in_node(j, n);
  p.vy = in_node(i, n) && in_seg(j, n);
  p.vz = in_node(i, n) && in_node(j, n);
  p.ox = p.vx ? (uint32_t)(j - 1) * n + i : 0u;
  p.oy = p.vy ? (uint32_t)j * n1 + (i - 1) : 0u;
  p.oz = p.vz ? (uint32_t)(j - 1) * n1 + (i - 1) : 0u;
  return p;
}

// FP64 operator on the integer pipe.  With the face and edge masses as the
// integer three-point weights [1, 4, 1] (1/6 and 1/36 folded into the
// coefficients), K u and M u have integer coefficients, so for u in fixed
// point (u * 2^s truncated to int64, max |u| 2^s < 2^55) both are computed
// exactly in int64: circulations stay below 2^57, face masses below 2^60, the
// four-face sums and the 3x3 edge masses below 2^62.  Only the final
// combination cK K u + cM M u and g - (...) run in FP64 (about 9 FP64
// instructions per lattice point instead of about 60), which matters on a part
// whose FP64 rate is 1/64 of its FP32 rate.  The scale comes from max |u| of
// each right-hand side (k_absmax); the truncation error is below
// 2^-54 max |u| per entry.
// (to_fixed and fixed_to_double: fpbits.cuh)

// sum over the 32 lanes of a warp (the same in every lane)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// max |x_r| of every right-hand side, as the bit pattern of |x| (monotonic as
// an unsigned integer, with Inf and NaN above every finite value); out[r]
// must be 0 on entry
__global__ void __launch_bounds__(256) k_absmax(int64_t N, const double* __restrict__ x,
                                                unsigned long long* __restrict__ out) {
  pdl_start();
  const double* xr = x + (int64_t)blockIdx.y * N;
  unsigned long long m = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(xr[e]) & 0x7FFFFFFFFFFFFFFFull;
    m = b > m ? b : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out + blockIdx.y, m);
}

// T: vector type (float / double); S: arithmetic type of the stencil (T, or
// long long for the fixed-point FP64 operator, which needs umax).  FLD: the
// curl-curl coefficient is constant per hexahedron (acell, n^3 values, cell
// (i, j, k) at (k n + j) n + i; cK = h times the pencil's factor): the face
// mass along the normal then weighs each of the two cells beside a face by its
// own coefficient, alpha_lo (c_lo + 2 c) + alpha_hi (2 c + c_hi) over 6, which
// is alpha (c_lo + 4 c + c_hi) / 6 for a constant one.
// pq (fixed-point FP64 apply only, optional): the CTA's sum of u_e y_e over
// its outputs, the block partial sums of u.(A u) for the PCG's curvature
// p.q, at pq[2 (rhs nb + b)] (second slot 0; b the CTA's index within its
// right-hand side, nb = gridDim.x gridDim.y z chunks), the layout of k_dot2
template <typename T, typename S, bool FLD = false>
__global__ void __launch_bounds__(kTX * kTY) k_stencil_stream(int n, int KZ, T cK, T cM, const T* __restrict__ u,
                                                              const T* __restrict__ g, T* __restrict__ y,
                                                              const unsigned long long* __restrict__ umax,
                                                              const T* __restrict__ acell = nullptr,
                                                              double* __restrict__ pq = nullptr) {
  pdl_start();
  static_assert(sizeof(S) == sizeof(T), "staged planes hold T and are read as S");
  constexpr bool FX = !std::is_same<S, T>::value;
  static_assert(!(FX && FLD), "the coefficient field runs in the vector type's own arithmetic");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* Ur = reinterpret_cast<S*>(smem_raw);  // [4 ring slots][x, y, z][kP]
  S* Cx = Ur + 12 * kP;                    // circulations of the current step
  S* Cy = Cx + kP;
  S* Cz = Cy + kP;
  T* Gr = reinterpret_cast<T*>(Cz + kP);   // [3 ring slots][x, y, z][kTP]
  T* Ar = Gr + 9 * kTP;                    // FLD: [4 ring slots][kP] cell coefficients
  const uint32_t n1 = n - 1, N3 = (uint32_t)n * n1 * n1;  // offsets within one right-hand side fit in 32 bits
  // grid z = (z chunks) x (right-hand sides); each right-hand side is a
  // contiguous canonical vector
  const int nzc = (n + KZ - 1) / KZ;
  const int rhs = blockIdx.z / nzc;
  u += (int64_t)rhs * 3 * N3;
  y += (int64_t)rhs * 3 * N3;
  if (g) g += (int64_t)rhs * 3 * N3;
  const int i0 = blockIdx.x * kTX, j0 = blockIdx.y * kTY, k0 = (blockIdx.z - rhs * nzc) * KZ;
  const int T_out = min(KZ, n - k0);  // output planes k0 .. k0 + T_out - 1
  const int tid = threadIdx.y * kTX + threadIdx.x;
  // fixed point: u 2^fs with max |u| 2^fs < 2^55; results carry 2^-fs
  int fs = 0;
  T cKo = cK * T(1.0 / 6.0), cMo = cM * T(1.0 / 36.0);  // three-point weights [1, 4, 1]
  if constexpr (FX) {
    const unsigned long long mb = umax[rhs];
    const int E = (int)((mb >> 52) & 0x7FF);  // max |u| < 2^(E - 1022)
    fs = mb == 0 ? 0 : 55 - (E - 1022);
    cKo = ldexp(cKo, -fs);
    cMo = ldexp(cMo, -fs);
    if (mb >= 0x7FF0000000000000ull) {  // Inf or NaN in u: the product is not finite
      fs = 0;
      cKo = cMo = T(NAN);
    }
  }
  // staged positions of this thread: q = tid and q = tid + kTP (when < kP)
  const int qa = tid, qb = tid + kTP;
  const bool has_b = qb < kP;
  const PlanePos pa = plane_pos(n, i0 + qa % kPX - 1, j0 + qa / kPX - 1);
  const PlanePos pb = plane_pos(n, i0 + qb % kPX - 1, j0 + qb / kPX - 1);
  const PlanePos pg = plane_pos(n, i0 + threadIdx.x, j0 + threadIdx.y);  // this thread's output column
  // plane terms of the global offsets of plane k (used only when valid)
  auto px = [&](int k) { return (uint32_t)(k - 1) * n1 * n; };
  auto py = [&](int k) { return N3 + (uint32_t)(k - 1) * n * n1; };
  auto pz = [&](int k) { return 2u * N3 + (uint32_t)k * n1 * n1; };
  auto stage_pos = [&](S* Sp, int q, const PlanePos& p, int k, bool kn, bool ks) {
    const bool vx = p.vx && kn, vy = p.vy && kn, vz = p.vz && ks;
    T* St = reinterpret_cast<T*>(Sp);
    cp_async_elem(St + q, u + (vx ? px(k) + p.ox : 0u), vx, u);
    cp_async_elem(St + kP + q, u + (vy ? py(k) + p.oy : 0u), vy, u);
    cp_async_elem(St + 2 * kP + q, u + (vz ? pz(k) + p.oz : 0u), vz, u);
  };
  // stage u on plane k, [i0-1, i0+TX] x [j0-1, j0+TY], into ring slot `slot`
  auto stage_u = [&](int k, int slot) {
    S* Sp = Ur + slot * 3 * kP;
    const bool kn = in_node(k, n), ks = in_seg(k, n);
    stage_pos(Sp, qa, pa, k, kn, ks);
    if (has_b) stage_pos(Sp, qb, pb, k, kn, ks);
  };
  // fixed point: this thread's own staged values of ring slot `slot`,
  // converted in place once its copies have landed
  auto convert_own = [&](int slot) {
    if constexpr (FX) {
      S* Sp = Ur + slot * 3 * kP;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Sp[c * kP + qa] = to_fixed(reinterpret_cast<const double*>(Sp)[c * kP + qa], fs);
        if (has_b) Sp[c * kP + qb] = to_fixed(reinterpret_cast<const double*>(Sp)[c * kP + qb], fs);
      }
    }
  };
  // stage g on plane k of the tile into ring slot `slot`
  auto stage_g = [&](int k, int slot) {
    T* Sg = Gr + slot * 3 * kTP;
    const bool kn = in_node(k, n), ks = in_seg(k, n);
    const bool vx = pg.vx && kn, vy = pg.vy && kn, vz = pg.vz && ks;
    cp_async_elem(Sg + tid, g + (vx ? px(k) + pg.ox : 0u), vx, g);
    cp_async_elem(Sg + kTP + tid, g + (vy ? py(k) + pg.oy : 0u), vy, g);
    cp_async_elem(Sg + 2 * kTP + tid, g + (vz ? pz(k) + pg.oz : 0u), vz, g);
  };
  // FLD: the coefficients of the cells of plane c (the hexahedra between
  // node planes c and c + 1) at the staged positions, cell plane p of the
  // chunk (c = k0 - 1 + p) in ring slot p % 4; zero outside the box (those
  // cells only meet faces whose circulation is zero)
  auto stage_a = [&](int c, int slot) {
    if constexpr (FLD) {
      T* Sa = Ar + slot * kP;
      const bool kc = (unsigned)c < (unsigned)n;
      auto one = [&](int qq) {
        const int ci = i0 + qq % kPX - 1, cj = j0 + qq / kPX - 1;
        const bool v = kc && (unsigned)ci < (unsigned)n && (unsigned)cj < (unsigned)n;
        cp_async_elem(Sa + qq, acell + (v ? ((uint32_t)c * n + (uint32_t)cj) * n + (uint32_t)ci : 0u), v, acell);
      };
      one(qa);
      if (has_b) one(qb);
    }
  };
  // u plane p of the chunk is z = k0 - 1 + p, held in ring slot p % 4; the
  // copies run two planes ahead of use (planes 0 and 1, and cell plane 0,
  // before the first step; one commit group per step)
  stage_u(k0 - 1, 0);
  stage_a(k0 - 1, 0);
  asm volatile("cp.async.commit_group;" ::: "memory");
  stage_u(k0, 1);
  asm volatile("cp.async.commit_group;" ::: "memory");

  const int a = threadIdx.x + 1, b = threadIdx.y + 1;
  const int q = b * kPX + a;
  auto f3 = [&](S m, S c0, S p1) { return (m + p1) + S(4) * c0; };
  // coefficient planes of the current step (FLD): cells of planes k - 1, k
  const T* Aprev = Ar;
  const T* Acur = Ar;
  // face mass along x / y of the current plane at (a,b) and its neighbours
  auto Xf = [&](int r) -> S {
    if constexpr (FLD) return Acur[r - 1] * (Cx[r - 1] + S(2) * Cx[r]) + Acur[r] * (S(2) * Cx[r] + Cx[r + 1]);
    else return f3(Cx[r - 1], Cx[r], Cx[r + 1]);
  };
  auto Yf = [&](int r) -> S {
    if constexpr (FLD)
      return Acur[r - kPX] * (Cy[r - kPX] + S(2) * Cy[r]) + Acur[r] * (S(2) * Cy[r] + Cy[r + kPX]);
    else return f3(Cy[r - kPX], Cy[r], Cy[r + kPX]);
  };
  // face mass along z at the face plane k between the cells (r, k-1) and (r, k)
  auto Zf = [&](int r, S m, S c0, S p1) -> S {
    if constexpr (FLD) return Aprev[r] * (m + S(2) * c0) + Acur[r] * (S(2) * c0 + p1);
    else return f3(m, c0, p1);
  };
  // rolling state: Cz at (a,b), (a,b-1), (a-1,b) and the in-plane edge-mass
  // rows of x- and y-edges, for planes k-1 (0) and k (1); Xf, Yf of plane k-1
  S cz0[3] = {S(0), S(0), S(0)}, cz1[3] = {S(0), S(0), S(0)};
  S rx0 = S(0), rx1 = S(0), ry0 = S(0), ry1 = S(0), yf_prev = S(0), xf_prev = S(0);
  double pqv = 0.0;  // pq: this thread's sum of u_e y_e
  // the circulation positions of this thread (fixed): neighbours staged?
  const bool ha_a = qa % kPX + 1 < kPX, hb_a = qa / kPX + 1 < kPY;
  const bool ha_b = qb % kPX + 1 < kPX, hb_b = qb / kPX + 1 < kPY;
  // y = g - (cK K u + cM M u) (or cK K u + cM M u) of one edge from its
  // integer-weighted sums kv, mv
  auto combine = [&](S kv, S mv, const T* Gp) -> T {
    T kd, md;
    if constexpr (FX) {
      kd = fixed_to_double(kv);
      md = fixed_to_double(mv);
    } else {
      kd = kv;
      md = mv;
    }
    if (g) return fma(-cMo, md, fma(-cKo, kd, *Gp));
    return fma(cMo, md, cKo * kd);
  };
  // step t forms the circulations of the current plane k0 + t (x- and
  // y-normal faces, t >= -1), those of the z-normal faces on the next plane
  // k0 + t + 1 and the next plane's edge-mass rows; outputs for t >= 0
  for (int t = -2; t < T_out; ++t) {
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // all but the newest group
    convert_own((t + 2) % 4);
    __syncthreads();  // u plane t+2, g(t) and cell plane t+1 landed; step t-1 is done with the rings
    if (t + 3 <= T_out) stage_u(k0 + t + 3, (t + 4) % 4);                 // u plane p = t + 4
    if (g && t + 2 < T_out) stage_g(k0 + t + 2, (t + 2) % 3);
    if (FLD && t + 3 <= T_out) stage_a(k0 + t + 2, (t + 3) % 4);         // cell plane p = t + 3
    asm volatile("cp.async.commit_group;" ::: "memory");
    const S* Uc = Ur + ((t + 5) % 4) * 3 * kP;  // plane k0 + t
    const S* Un = Ur + ((t + 2) % 4) * 3 * kP;  // plane k0 + t + 1
    if constexpr (FLD) {
      Aprev = Ar + ((t + 4) % 4) * kP;  // cell plane k0 + t - 1 (p = t)
      Acur = Ar + ((t + 5) % 4) * kP;   // cell plane k0 + t (p = t + 1)
    }
    auto circ = [&](int r, bool ha, bool hb) {
      if (t >= -1) {
        // cx(i,j,k) = uz(i,j+1,k) - uz(i,j,k) - uy(i,j,k+1) + uy(i,j,k)
        Cx[r] = hb ? Uc[2 * kP + r + kPX] - Uc[2 * kP + r] - Un[kP + r] + Uc[kP + r] : S(0);
        // cy(i,j,k) = ux(i,j,k+1) - ux(i,j,k) - uz(i+1,j,k) + uz(i,j,k)
        Cy[r] = ha ? Un[r] - Uc[r] - Uc[2 * kP + r + 1] + Uc[2 * kP + r] : S(0);
      }
      // cz(i,j,k+1) = uy(i+1,j,k+1) - uy(i,j,k+1) - ux(i,j+1,k+1) + ux(i,j,k+1)
      Cz[r] = (ha && hb) ? Un[kP + r + 1] - Un[kP + r] - Un[r + kPX] + Un[r] : S(0);
    };
    circ(qa, ha_a, hb_a);
    if (has_b) circ(qb, ha_b, hb_b);
    __syncthreads();
    const S cz2[3] = {Cz[q], Cz[q - kPX], Cz[q - 1]};
    const S rx2 = f3(Un[q - kPX], Un[q], Un[q + kPX]);               // x-edges vary in y
    const S ry2 = f3(Un[kP + q - 1], Un[kP + q], Un[kP + q + 1]);    // y-edges vary in x
    if (t >= -1) {
      const S yf = Yf(q), xf = Xf(q);
      if (t >= 0) {
        const int k = k0 + t;
        const bool kn = in_node(k, n), ks = in_seg(k, n);
        const T* G = Gr + (t % 3) * 3 * kTP;
        const S zf = Zf(q, cz0[0], cz1[0], cz2[0]);          // Zf(a, b, k)
        const S zf_b = Zf(q - kPX, cz0[1], cz1[1], cz2[1]);  // Zf(a, b-1, k)
        const S zf_a = Zf(q - 1, cz0[2], cz1[2], cz2[2]);    // Zf(a-1, b, k)
        // store one output; with pq also add u_e y_e (u_e read back in
        // FP64: the staged copy is in fixed point)
        auto put = [&](uint32_t o, T v) {
          y[o] = v;
          if constexpr (FX)
            if (pq) pqv = fma((double)u[o], (double)v, pqv);
        };
        if (pg.vx && kn) put(px(k) + pg.ox, combine((yf_prev - yf) + (zf - zf_b), f3(rx0, rx1, rx2), G + tid));
        if (pg.vy && kn) put(py(k) + pg.oy, combine((zf_a - zf) + (xf - xf_prev), f3(ry0, ry1, ry2), G + kTP + tid));
        if (pg.vz && ks) {
          const S* Uz = Uc + 2 * kP;
          const S kv = (Xf(q - kPX) - xf) + (yf - Yf(q - 1));
          const S mz = f3(f3(Uz[q - kPX - 1], Uz[q - 1], Uz[q + kPX - 1]), f3(Uz[q - kPX], Uz[q], Uz[q + kPX]),
                          f3(Uz[q - kPX + 1], Uz[q + 1], Uz[q + kPX + 1]));
          put(pz(k) + pg.oz, combine(kv, mz, G + 2 * kTP + tid));
        }
      }
      yf_prev = yf;
      xf_prev = xf;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cz0[c] = cz1[c];
      cz1[c] = cz2[c];
    }
    rx0 = rx1; rx1 = rx2;
    ry0 = ry1; ry1 = ry2;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if constexpr (FX) {
    if (pq) {  // one warp per row of the block (kTX = 32)
      __shared__ double pq_rows[kTY];
      const double w = warp_sum(pqv);
      if (threadIdx.x == 0) pq_rows[threadIdx.y] = w;
      __syncthreads();
      if (tid == 0) {
        double sum = 0.0;
#pragma unroll
        for (int r = 0; r < kTY; ++r) sum += pq_rows[r];
        const int64_t nb = (int64_t)gridDim.x * gridDim.y * nzc;
        const int64_t b = ((int64_t)(blockIdx.z - rhs * nzc) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        pq[2 * (rhs * nb + b)] = sum;
        pq[2 * (rhs * nb + b) + 1] = 0.0;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Grid transfer (Sec. 3.1).  Prolongation = natural injection N_{k-1} ->
// N_k: along a coarse edge both fine halves take its value; across it the
// coarse hat is linear (weight 1 at the coarse node, 1/2 one fine node away).
// Restriction is the transpose.
// ---------------------------------------------------------------------------
// One thread per lattice point (i, j, k) of the output mesh handles the x-,
// y- and z-edge that start there (when they are interior); blocks of 32 x 8
// threads run along i, the grid's z index is k.
// zc (optional): the coarse solution, set to 0 at the same entries (the
// V-cycle recursion starts the coarse level from z = 0)
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(int nf, const T* __restrict__ rf, T* __restrict__ gc,
                                                  T* __restrict__ zc) {
  pdl_start();
  const int nc = nf / 2;
  const int rhs = blockIdx.z / nc;
  const int I = blockIdx.x * 32 + threadIdx.x, J = blockIdx.y * 8 + threadIdx.y, K = blockIdx.z - rhs * nc;
  if (I >= nc || J >= nc) return;
  const int64_t N3c = (int64_t)nc * (nc - 1) * (nc - 1);
  const int64_t N3f = (int64_t)nf * (nf - 1) * (nf - 1);
  rf += (int64_t)rhs * 3 * N3f;
  gc += (int64_t)rhs * 3 * N3c;
  if (zc) {
    zc += (int64_t)rhs * 3 * N3c;
    if (in_node(J, nc) && in_node(K, nc)) zc[off_x(nc, I, J, K)] = T(0);
    if (in_node(I, nc) && in_node(K, nc)) zc[N3c + off_y(nc, I, J, K)] = T(0);
    if (in_node(I, nc) && in_node(J, nc)) zc[2 * N3c + off_z(nc, I, J, K)] = T(0);
  }
  const T w[3] = {T(0.5), T(1), T(0.5)};
  // coarse x-edge (I, J, K): fine x-edges 2I+a, 2J+b, 2K+c with weight w_b w_c
  if (in_node(J, nc) && in_node(K, nc)) {
    T s = T(0);
#pragma unroll
    for (int c = -1; c <= 1; ++c)
#pragma unroll
      for (int b = -1; b <= 1; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) s += w[b + 1] * w[c + 1] * __ldg(rf + off_x(nf, 2 * I + a, 2 * J + b, 2 * K + c));
    gc[off_x(nc, I, J, K)] = s;
  }
  if (in_node(I, nc) && in_node(K, nc)) {
    T s = T(0);
#pragma unroll
    for (int c = -1; c <= 1; ++c)
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = -1; b <= 1; ++b)
          s += w[b + 1] * w[c + 1] * __ldg(rf + N3f + off_y(nf, 2 * I + b, 2 * J + a, 2 * K + c));
    gc[N3c + off_y(nc, I, J, K)] = s;
  }
  if (in_node(I, nc) && in_node(J, nc)) {
    T s = T(0);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = -1; c <= 1; ++c)
#pragma unroll
        for (int b = -1; b <= 1; ++b)
          s += w[b + 1] * w[c + 1] * __ldg(rf + 2 * N3f + off_z(nf, 2 * I + b, 2 * J + c, 2 * K + a));
    gc[2 * N3c + off_z(nc, I, J, K)] = s;
  }
}

// Prolongation z_f += P z_c, one thread per fine lattice point (i, j, k)
// adding into its x-, y- and z-edge (each a plain coalesced read-modify-write
// of the thread's own entry, so no atomics).  Along a coarse edge both fine
// halves take its value; across it the coarse hat is linear (fine node 2P:
// weight 1 at coarse node P; fine node 2P + 1: weight 1/2 at P and P + 1),
// coarse boundary nodes carrying 0.  Neighbouring threads read the same few
// coarse values, which the L1 serves.
template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(int nf, const T* __restrict__ zc, T* __restrict__ zf) {
  pdl_start();
  const int rhs = blockIdx.z / nf;
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z - rhs * nf;
  if (i >= nf || j >= nf) return;
  const int nc = nf >> 1, n1 = nf - 1, c1 = nc - 1;
  const int64_t N3c = (int64_t)nc * c1 * c1, N3f = (int64_t)nf * n1 * n1;
  const T* cx = zc + rhs * 3 * N3c;
  const T* cy = cx + N3c;
  const T* cz = cy + N3c;
  T* fx = zf + rhs * 3 * N3f;
  T* fy = fx + N3f;
  T* fz = fy + N3f;
  const int I = i >> 1, J = j >> 1, K = k >> 1, di = i & 1, dj = j & 1, dk = k & 1;
  // x-edge: segment i, nodes (j, k); y-edge: segment j, nodes (i, k); z-edge:
  // segment k, nodes (i, j).  Offsets within one direction fit 32 bits
  // (n <= 1024); the coarse neighbours are constant strides from one base.
  const bool vx = in_node(j, nf) && in_node(k, nf);
  const bool vy = in_node(i, nf) && in_node(k, nf);
  const bool vz = in_node(i, nf) && in_node(j, nf);
  const int ofx = ((k - 1) * n1 + (j - 1)) * nf + i;
  const int ofy = ((k - 1) * nf + j) * n1 + (i - 1);
  const int ofz = (k * n1 + (j - 1)) * n1 + (i - 1);
  // all loads (3 fine, up to 12 coarse) are issued before the first store
  const T ax = vx ? fx[ofx] : T(0), ay = vy ? fy[ofy] : T(0), az = vz ? fz[ofz] : T(0);
  // interior coarse nodes P (and P + 1 where the fine node is odd)
  const bool I0 = in_node(I, nc), J0 = in_node(J, nc), K0 = in_node(K, nc);
  const bool I1 = di && in_node(I + 1, nc), J1 = dj && in_node(J + 1, nc), K1 = dk && in_node(K + 1, nc);
  const int ocx = ((K - 1) * c1 + (J - 1)) * nc + I;  // +nc: J + 1; +c1 nc: K + 1
  const int ocy = ((K - 1) * nc + J) * c1 + (I - 1);  // +1: I + 1; +nc c1: K + 1
  const int ocz = (K * c1 + (J - 1)) * c1 + (I - 1);  // +1: I + 1; +c1: J + 1
  auto ld = [](bool ok, const T* p) { return ok ? __ldg(p) : T(0); };
  const T x00 = ld(vx && J0 && K0, cx + ocx), x10 = ld(vx && J1 && K0, cx + ocx + nc),
          x01 = ld(vx && J0 && K1, cx + ocx + c1 * nc), x11 = ld(vx && J1 && K1, cx + ocx + nc + c1 * nc);
  const T y00 = ld(vy && I0 && K0, cy + ocy), y10 = ld(vy && I1 && K0, cy + ocy + 1),
          y01 = ld(vy && I0 && K1, cy + ocy + nc * c1), y11 = ld(vy && I1 && K1, cy + ocy + 1 + nc * c1);
  const T z00 = ld(vz && I0 && J0, cz + ocz), z10 = ld(vz && I1 && J0, cz + ocz + 1),
          z01 = ld(vz && I0 && J1, cz + ocz + c1), z11 = ld(vz && I1 && J1, cz + ocz + 1 + c1);
  // value at fine across-nodes (2P + d1, 2Q + d2) from the coarse values at
  // (P + a, Q + b); entries with a > d1 or b > d2 are 0 and unused
  auto lerp = [](T v00, T v10, T v01, T v11, int d1, int d2) -> T {
    const T v0 = d1 ? T(0.5) * (v00 + v10) : v00;
    const T v1 = d1 ? T(0.5) * (v01 + v11) : v01;
    return d2 ? T(0.5) * (v0 + v1) : v0;
  };
  if (vx) fx[ofx] = ax + lerp(x00, x10, x01, x11, dj, dk);
  if (vy) fy[ofy] = ay + lerp(y00, y10, y01, y11, di, dk);
  if (vz) fz[ofz] = az + lerp(z00, z10, z01, z11, di, dj);
}

// The same prolongation, one thread per coarse cell (I, J, K) updating the
// 24 fine edges of its
// 2 x 2 x 2 block of fine lattice points (2I + di, 2J + dj, 2K + dk) from 12
// coarse values loaded once; the fine x-edge pair (2I, 2I+1) is one
// 2-element access.  Eight times fewer threads than the per-fine-point form,
// whose index arithmetic it shares among 24 edges: the faster form on the
// largest grids, the per-fine-point one on the smaller.
template <typename T>
struct Vec2;
template <>
struct Vec2<float> { using type = float2; };
template <>
struct Vec2<double> { using type = double2; };

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add_cell(int nf, const T* __restrict__ zc, T* __restrict__ zf) {
  pdl_start();
  const int nc = nf / 2;
  const int rhs = blockIdx.z / nc;
  const int I = blockIdx.x * 32 + threadIdx.x, J = blockIdx.y * 8 + threadIdx.y, K = blockIdx.z - rhs * nc;
  if (I >= nc || J >= nc) return;
  const int64_t N3c = (int64_t)nc * (nc - 1) * (nc - 1);
  const int64_t N3f = (int64_t)nf * (nf - 1) * (nf - 1);
  zc += (int64_t)rhs * 3 * N3c;
  zf += (int64_t)rhs * 3 * N3f;
  auto cin = [&](int p) { return in_node(p, nc); };  // interior coarse node
  T X[2][2], Y[2][2], Z[2][2];  // [first across node offset][second across node offset]
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      X[a][b] = cin(J + a) && cin(K + b) ? __ldg(zc + off_x(nc, I, J + a, K + b)) : T(0);
      Y[a][b] = cin(I + a) && cin(K + b) ? __ldg(zc + N3c + off_y(nc, I + a, J, K + b)) : T(0);
      Z[a][b] = cin(I + a) && cin(J + b) ? __ldg(zc + 2 * N3c + off_z(nc, I + a, J + b, K)) : T(0);
    }
  // value at fine across-offsets (d1, d2) from the 2 x 2 coarse values V
  auto lerp = [](const T (&V)[2][2], int d1, int d2) -> T {
    const T v0 = d1 ? T(0.5) * (V[0][0] + V[1][0]) : V[0][0];
    const T v1 = d1 ? T(0.5) * (V[0][1] + V[1][1]) : V[0][1];
    return d2 ? T(0.5) * (v0 + v1) : v0;
  };
  using T2 = typename Vec2<T>::type;
#pragma unroll
  for (int d2 = 0; d2 < 2; ++d2)
#pragma unroll
    for (int d1 = 0; d1 < 2; ++d1) {
      // x-edges (2I, 2I+1) at nodes (2J + d1, 2K + d2): fine node 0 is on the boundary
      if ((d1 || J >= 1) && (d2 || K >= 1)) {
        const T v = lerp(X, d1, d2);
        T2* p = reinterpret_cast<T2*>(zf + off_x(nf, 2 * I, 2 * J + d1, 2 * K + d2));
        T2 w = *p;
        w.x += v;
        w.y += v;
        *p = w;
      }
      // y-edges (segments 2J, 2J+1) at nodes (2I + d1, 2K + d2)
      if ((d1 || I >= 1) && (d2 || K >= 1)) {
        const T v = lerp(Y, d1, d2);
        zf[N3f + off_y(nf, 2 * I + d1, 2 * J, 2 * K + d2)] += v;
        zf[N3f + off_y(nf, 2 * I + d1, 2 * J + 1, 2 * K + d2)] += v;
      }
      // z-edges (segments 2K, 2K+1) at nodes (2I + d1, 2J + d2)
      if ((d1 || I >= 1) && (d2 || J >= 1)) {
        const T v = lerp(Z, d1, d2);
        zf[2 * N3f + off_z(nf, 2 * I + d1, 2 * J + d2, 2 * K)] += v;
        zf[2 * N3f + off_z(nf, 2 * I + d1, 2 * J + d2, 2 * K + 1)] += v;
      }
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
  pdl_start();
  const int nc = n / 2;
  const int64_t NT = (int64_t)nc * nc * nc;
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  r += (int64_t)blockIdx.y * 3 * N3;
  z += (int64_t)blockIdx.y * 3 * N3;
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

// Dense patch solves on CUDA cores: z += eta * D r_p for every patch of one
// family, D = J_D A_D^{-1} J_D^t (nloc x nloc, symmetric) staged in shared
// memory, PB patches per pass; overlapping patches accumulate with atomics.
// A family is a lattice of boxes of cells (vertex patches: 4x4x4 around each
// interior coarse vertex; edge patches: 2 cells along a coarse edge x 4 x 4
// across); patch (pa, pb, pc) has its box origin at 2 (pa, pb, pc) - shift,
// and its local edges follow the canonical numbering of that box.
template <typename T, int PB>
__global__ void __launch_bounds__(128) k_patch_dense(int n, PatchFamily fam, const T* __restrict__ D, T eta,
                                                     const T* __restrict__ r, T* __restrict__ z) {
  pdl_start();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nl = fam.nloc;
  T* Ds = reinterpret_cast<T*>(smem_raw);          // nl * nl
  T* Rs = Ds + nl * nl;                            // nl * PB
  int* loc = reinterpret_cast<int*>(Rs + nl * PB); // packed (d, i, j, k) of each local edge
  const int64_t NP = (int64_t)fam.np[0] * fam.np[1] * fam.np[2];
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  r += (int64_t)blockIdx.y * 3 * N3;
  z += (int64_t)blockIdx.y * 3 * N3;
  for (int q = threadIdx.x; q < nl * nl; q += blockDim.x) Ds[q] = D[q];
  const int bx = fam.b[0], by = fam.b[1], bz = fam.b[2];
  const int cx = bx * (by - 1) * (bz - 1), cy = (bx - 1) * by * (bz - 1);
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    int d, i, j, k, e = l;
    if (e < cx) {
      d = 0; i = e % bx; j = (e / bx) % (by - 1) + 1; k = e / (bx * (by - 1)) + 1;
    } else if ((e -= cx) < cy) {
      d = 1; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % by; k = e / ((bx - 1) * by) + 1;
    } else {
      e -= cy;
      d = 2; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % (by - 1) + 1; k = e / ((bx - 1) * (by - 1));
    }
    loc[l] = (((d * 16 + i) * 16 + j) * 16) + k;
  }
  auto gidx_of = [&](int64_t P, int l) {
    const int pa = (int)(P % fam.np[0]) + fam.p0[0];
    const int pb = (int)((P / fam.np[0]) % fam.np[1]) + fam.p0[1];
    const int pc = (int)(P / ((int64_t)fam.np[0] * fam.np[1])) + fam.p0[2];
    const int c = loc[l];
    const int d = c >> 12, i = (c >> 8) & 15, j = (c >> 4) & 15, k = c & 15;
    return edge_gidx(n, d, fam.stride * pa - fam.shift[0] + i, fam.stride * pb - fam.shift[1] + j,
                     fam.stride * pc - fam.shift[2] + k);
  };
  for (int64_t base = (int64_t)blockIdx.x * PB; base < NP; base += (int64_t)gridDim.x * PB) {
    __syncthreads();
    for (int q = threadIdx.x; q < nl * PB; q += blockDim.x) {
      const int p = q / nl, l = q % nl;
      const int64_t P = base + p;
      Rs[l * PB + p] = P < NP ? __ldg(r + gidx_of(P, l)) : T(0);
    }
    __syncthreads();
    for (int row = threadIdx.x; row < nl; row += blockDim.x) {
      T acc[PB];
#pragma unroll
      for (int p = 0; p < PB; ++p) acc[p] = T(0);
      for (int c = 0; c < nl; ++c) {
        const T dv = Ds[c * nl + row];
#pragma unroll
        for (int p = 0; p < PB; ++p) acc[p] += dv * Rs[c * PB + p];
      }
#pragma unroll
      for (int p = 0; p < PB; ++p)
        if (base + p < NP) atomicAdd(z + gidx_of(base + p, row), eta * acc[p]);
    }
  }
}

// The FP64 dense patch solves in double-float arithmetic on the FP32 pipe.
// This part's FP64 rate is about 1/64 of its FP32 rate, and the dense
// 108 x 108 patch products bound the FP64 V-cycle.  Every value is split
// into a pair of floats (hi = fl(v), lo = fl(v - hi), about 48 significant
// bits together); a product term d r is formed as hi*hi (rounded) plus its
// exact rounding error (fma) plus the two cross terms, and added to a
// running float sum with an error-free two-sum whose error joins a float
// compensation; every kFold terms that pair is folded the same way into a
// running pair, converted to FP64 once at the end (FP64 instructions run at
// 1/64 of the FP32 rate here, so none sits in the inner loops).  The residual block of a pass is scaled by a power of two so
// that its largest entry is near 1 (the float exponent range then holds
// every useful entry), and the result is scaled back.  The sums stay within
// about 1e-14 of the FP64 ones relative to the largest term.
constexpr int kFold = 16;
constexpr int kDfThreads = 256;             // two thread halves, one row each
constexpr int kPBdf = 16;                   // patches per pass: 8 per half

// lin_d(i, j, k): the affine part of edge_gidx for direction d, so that
// edge_gidx(n, d, o + (i, j, k)) = edge_gidx(n, d, o) + lin_d(i, j, k)
__device__ __forceinline__ int edge_lin(int n, int d, int i, int j, int k) {
  return d == 0 ? i + n * j + n * (n - 1) * k : d == 1 ? i + (n - 1) * j + n * (n - 1) * k
                                                     : i + (n - 1) * j + (n - 1) * (n - 1) * k;
}

// v 2^-ex as a pair of floats hi + lo on the integer pipe (no FP64
// instruction): hi takes the top 24 bits of the significand, lo the next 24
// (the last 5 of 53 are dropped: relative error below 2^-47 of |v|); v whose
// scaled magnitude is below 2^-100 (the pass maximum is scaled into [1, 2))
// gives 0; Inf and NaN give NaN
__device__ __forceinline__ void split_scaled(double v, int ex, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const int eu = e - 1023 - ex;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned r29 = (unsigned)(m & 0x1FFFFFFFull);
  const int top = 31 - __clz(r29 | 1u);  // leading one of the low 29 bits
  const int el = eu - 52 + top;
  const unsigned ml = top >= 23 ? r29 >> (top - 23) : r29 << (23 - top);
  const bool tiny = e == 0 || eu < -100;
  hi = tiny ? 0.f : __uint_as_float(sign | ((unsigned)(eu + 127) << 23) | ((unsigned)(m >> 29) & 0x7FFFFFu));
  lo = (tiny || r29 == 0u || el < -126) ? 0.f : __uint_as_float(sign | ((unsigned)(el + 127) << 23) | (ml & 0x7FFFFFu));
  if (e == 0x7FF) hi = lo = __uint_as_float(0x7FC00000u);
}

// a float as a double on the integer pipe: normal floats and zeros exactly,
// subnormals as zero, Inf and NaN as NaN
__device__ __forceinline__ double float_bits_to_double(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned ef = (u >> 23) & 0xFFu;
  const unsigned long long bits =
      ef == 0u ? s
               : (ef == 0xFFu ? 0x7FF8000000000000ull
                              : s | ((unsigned long long)(ef + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29));
  return __longlong_as_double((long long)bits);
}

__global__ void __launch_bounds__(kDfThreads, 2) k_patch_dense_df(int n, PatchFamily fam, const double* __restrict__ D,
                                                               double eta, const double* __restrict__ r,
                                                               double* __restrict__ z) {
  pdl_start();
  constexpr int H = kPBdf / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nl = fam.nloc;
  const int nl2 = (nl * nl + 3) & ~3;               // keeps Rh, Rl 16-byte aligned
  float* Dh = reinterpret_cast<float*>(smem_raw);   // nl * nl
  float* Dl = Dh + nl2;
  float* Rh = Dl + nl2;                             // nl * kPBdf
  float* Rl = Rh + nl * kPBdf;
  unsigned* loff = reinterpret_cast<unsigned*>(Rl + nl * kPBdf);  // lin_d of each local edge, d in the top 2 bits
  long long* pbase = reinterpret_cast<long long*>(loff + ((nl + 1) & ~1));  // [kPBdf][3] edge_gidx of the origins
  unsigned* amax = reinterpret_cast<unsigned*>(pbase + 3 * kPBdf);
  const int64_t NP = (int64_t)fam.np[0] * fam.np[1] * fam.np[2];
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  r += (int64_t)blockIdx.y * 3 * N3;
  z += (int64_t)blockIdx.y * 3 * N3;
  {
    // the operator's float parts follow its FP64 entries (dense_stride)
    const float* hl = reinterpret_cast<const float*>(D + nl * nl);
    for (int q = threadIdx.x; q < nl * nl; q += blockDim.x) {
      Dh[q] = __ldg(hl + q);
      Dl[q] = __ldg(hl + nl * nl + q);
    }
  }
  const int bx = fam.b[0], by = fam.b[1], bz = fam.b[2];
  const int cx = bx * (by - 1) * (bz - 1), cy = (bx - 1) * by * (bz - 1);
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    int d, i, j, k, e = l;
    if (e < cx) {
      d = 0; i = e % bx; j = (e / bx) % (by - 1) + 1; k = e / (bx * (by - 1)) + 1;
    } else if ((e -= cx) < cy) {
      d = 1; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % by; k = e / ((bx - 1) * by) + 1;
    } else {
      e -= cy;
      d = 2; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % (by - 1) + 1; k = e / ((bx - 1) * (by - 1));
    }
    loff[l] = (unsigned)edge_lin(n, d, i, j, k) | ((unsigned)d << 30);
  }
  __syncthreads();
  const int half = threadIdx.x / 128, row = threadIdx.x % 128;
  const bool active = row < nl;
  const int my_off = active ? (int)(loff[row] & 0x3FFFFFFFu) : 0, my_d = active ? (int)(loff[row] >> 30) : 0;
  for (int64_t base = (int64_t)blockIdx.x * kPBdf; base < NP; base += (int64_t)gridDim.x * kPBdf) {
    // the origins of this pass's patches (one 64-bit division per patch)
    if (threadIdx.x < kPBdf * 3) {
      const int pp = threadIdx.x / 3, d = threadIdx.x % 3;
      const int64_t P = base + pp < NP ? base + pp : NP - 1;
      const int pa = (int)(P % fam.np[0]) + fam.p0[0];
      const int pb = (int)((P / fam.np[0]) % fam.np[1]) + fam.p0[1];
      const int pc = (int)(P / ((int64_t)fam.np[0] * fam.np[1])) + fam.p0[2];
      pbase[threadIdx.x] = edge_gidx(n, d, fam.stride * pa - fam.shift[0], fam.stride * pb - fam.shift[1],
                                     fam.stride * pc - fam.shift[2]);
    }
    if (threadIdx.x == 0) *amax = 0u;
    __syncthreads();
    // gather: thread (half, row) loads local edge `row` of the half's 8 patches;
    // m: the largest upper word of |r| (ordered like |r|, Inf and NaN on top)
    double rv[H];
    unsigned m = 0;
#pragma unroll
    for (int p = 0; p < H; ++p) {
      const int pp = half * H + p;
      rv[p] = active && base + pp < NP ? __ldg(r + pbase[3 * pp + my_d] + my_off) : 0.0;
      m = max(m, (unsigned)((unsigned long long)__double_as_longlong(rv[p]) >> 32) & 0x7FFFFFFFu);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax, m);
    __syncthreads();
    // 2^-ex brings the largest entry of the pass into [1, 2) (a pass of zeros
    // keeps ex = 0; Inf or NaN propagate as NaN)
    const unsigned mw = *amax;
    const int ex = mw == 0 ? 0 : (int)(mw >> 20) - 1023;
    if (active) {
#pragma unroll
      for (int p = 0; p < H; ++p) {
        float hi, lo;
        split_scaled(rv[p], ex, hi, lo);
        Rh[row * kPBdf + half * H + p] = hi;
        Rl[row * kPBdf + half * H + p] = lo;
      }
    }
    __syncthreads();
    if (active) {
      float ah[H], al[H], sh[H], sl[H];
#pragma unroll
      for (int p = 0; p < H; ++p) {
        ah[p] = al[p] = 0.f;
        sh[p] = sl[p] = 0.f;
      }
      for (int c0 = 0; c0 < nl; c0 += kFold) {
        const int c1 = c0 + kFold < nl ? c0 + kFold : nl;
        #pragma unroll 2
        for (int c = c0; c < c1; ++c) {
          const float dh = Dh[c * nl + row], dl = Dl[c * nl + row];
          const float4* rh4 = reinterpret_cast<const float4*>(Rh + c * kPBdf + half * H);
          const float4* rl4 = reinterpret_cast<const float4*>(Rl + c * kPBdf + half * H);
          const float4 h0 = rh4[0], h1 = rh4[1], l0 = rl4[0], l1 = rl4[1];
          const float rh[H] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
          const float rl[H] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
#pragma unroll
          for (int p = 0; p < H; ++p) {
            const float prod = __fmul_rn(dh, rh[p]);
            const float err = fmaf(dh, rh[p], -prod);               // exact: dh rh = prod + err
            const float low = fmaf(dh, rl[p], fmaf(dl, rh[p], err));
            const float t = __fadd_rn(sh[p], prod);                 // two-sum: sh + prod = t + e2 exactly
            const float bb = __fsub_rn(t, sh[p]);
            const float e2 = __fadd_rn(__fsub_rn(sh[p], __fsub_rn(t, bb)), __fsub_rn(prod, bb));
            sh[p] = t;
            sl[p] = __fadd_rn(sl[p], __fadd_rn(e2, low));
          }
        }
        // fold the chunk's pair into the running pair (ah, al) the same way
#pragma unroll
        for (int p = 0; p < H; ++p) {
          const float t = __fadd_rn(ah[p], sh[p]);
          const float bb = __fsub_rn(t, ah[p]);
          const float e2 = __fadd_rn(__fsub_rn(ah[p], __fsub_rn(t, bb)), __fsub_rn(sh[p], bb));
          ah[p] = t;
          al[p] = __fadd_rn(al[p], __fadd_rn(e2, sl[p]));
          sh[p] = sl[p] = 0.f;
        }
      }
      const double back = ldexp(eta, ex);
#pragma unroll
      for (int p = 0; p < H; ++p) {
        const int pp = half * H + p;
        if (base + pp < NP)
          atomicAdd(z + pbase[3 * pp + my_d] + my_off,
                    back * (float_bits_to_double(ah[p]) + float_bits_to_double(al[p])));
      }
    }
    __syncthreads();  // pbase, Rh, Rl are rewritten by the next pass
  }
}

// The whole smoother correction of eq. (Preconditioner P) for a small level
// in one launch on CUDA cores: CTAs [0, npb) take PB vertex patches each
// (every element of the dense 108 x 108 operator feeds PB patches from a
// register), the other CTAs take the 6 x 6 interior solves of 128 coarse
// elements each; both add into z with atomics (vertex patches contain
// element-interior edges).  The operator is
// copied into shared memory before the kernel waits for its predecessor (it
// is constant), so on levels with a few hundred patches a CTA's critical path
// is one gather, the product and the atomics.
template <int PB>
__global__ void __launch_bounds__(128) k_smooth_direct(int n, PatchFamily fam, const float* __restrict__ D,
                                                       const float* __restrict__ Ainv, float eta, int npb,
                                                       const float* __restrict__ r, float* __restrict__ z) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  constexpr int NL = 108;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ds = reinterpret_cast<float*>(smem_raw);  // NL x NL
  __shared__ float Rs[NL * PB];
  __shared__ unsigned loff[NL];
  __shared__ long long pbase[3 * PB];
  __shared__ float As[36];
  const int tid = threadIdx.x;
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  if ((int)blockIdx.x < npb) {
    // the operator (constant: copied before the wait for the previous kernel)
    {
      const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(Ds));
      const float4* src = reinterpret_cast<const float4*>(D);
      for (int q = tid; q < NL * NL / 4; q += blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16u * q), "l"(src + q) : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // local offsets of the 108 patch edges (independent of the previous kernel)
    if (tid < NL) {
      const int bx = fam.b[0], by = fam.b[1], bz = fam.b[2];
      const int cx = bx * (by - 1) * (bz - 1), cy = (bx - 1) * by * (bz - 1);
      int d, i, j, k, e = tid;
      if (e < cx) {
        d = 0; i = e % bx; j = (e / bx) % (by - 1) + 1; k = e / (bx * (by - 1)) + 1;
      } else if ((e -= cx) < cy) {
        d = 1; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % by; k = e / ((bx - 1) * by) + 1;
      } else {
        e -= cy;
        d = 2; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % (by - 1) + 1; k = e / ((bx - 1) * (by - 1));
      }
      loff[tid] = (unsigned)edge_lin(n, d, i, j, k) | ((unsigned)d << 30);
    }
    const int64_t NP = (int64_t)fam.np[0] * fam.np[1] * fam.np[2];
    const int64_t base = (int64_t)blockIdx.x * PB;
    if (tid < 3 * PB) {
      const int pp = tid / 3, d = tid % 3;
      const int64_t P = base + pp < NP ? base + pp : NP - 1;
      const int pa = (int)(P % fam.np[0]) + fam.p0[0];
      const int pb = (int)((P / fam.np[0]) % fam.np[1]) + fam.p0[1];
      const int pc = (int)(P / ((int64_t)fam.np[0] * fam.np[1])) + fam.p0[2];
      pbase[tid] = edge_gidx(n, d, fam.stride * pa - fam.shift[0], fam.stride * pb - fam.shift[1],
                             fam.stride * pc - fam.shift[2]);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    r += (int64_t)blockIdx.y * 3 * N3;
    z += (int64_t)blockIdx.y * 3 * N3;
    __syncthreads();
    for (int q = tid; q < NL * PB; q += blockDim.x) {
      const int pp = q / NL, l = q - pp * NL;
      const unsigned c = loff[l];
      Rs[l * PB + pp] = base + pp < NP ? __ldg(r + pbase[3 * pp + (int)(c >> 30)] + (int)(c & 0x3FFFFFFFu)) : 0.f;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    if (tid < NL) {
      float acc[PB];
#pragma unroll
      for (int p = 0; p < PB; ++p) acc[p] = 0.f;
#pragma unroll 4
      for (int c = 0; c < NL; ++c) {
        const float dv = Ds[c * NL + tid];
#pragma unroll
        for (int p = 0; p < PB; ++p) acc[p] = fmaf(dv, Rs[c * PB + p], acc[p]);
      }
      const unsigned c = loff[tid];
      const int d = (int)(c >> 30), off = (int)(c & 0x3FFFFFFFu);
#pragma unroll
      for (int p = 0; p < PB; ++p)
        if (base + p < NP) atomicAdd(z + pbase[3 * p + d] + off, eta * acc[p]);
    }
    return;
  }
  // interior spaces: one coarse element per thread
  if (tid < 36) As[tid] = __ldg(Ainv + tid);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  r += (int64_t)blockIdx.y * 3 * N3;
  z += (int64_t)blockIdx.y * 3 * N3;
  __syncthreads();
  const int nc = n / 2;
  const int64_t NT = (int64_t)nc * nc * nc;
  const int64_t t = (int64_t)(blockIdx.x - npb) * blockDim.x + tid;
  if (t >= NT) return;
  const int I = (int)(t % nc), J = (int)((t / nc) % nc), K = (int)(t / ((int64_t)nc * nc));
  int64_t g[6];
  int q = 0;
  for (int d = 0; d < 3; ++d)
    for (int s2 = 0; s2 < 2; ++s2) {
      int p[3] = {2 * I + 1, 2 * J + 1, 2 * K + 1};
      p[d] = (d == 0 ? 2 * I : d == 1 ? 2 * J : 2 * K) + s2;
      g[q++] = edge_gidx(n, d, p[0], p[1], p[2]);
    }
  float rv[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) rv[a] = __ldg(r + g[a]);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    float sum = 0.f;
#pragma unroll
    for (int b = 0; b < 6; ++b) sum = fmaf(As[a * 6 + b], rv[b], sum);
    atomicAdd(z + g[a], eta * sum);
  }
}

// Vertex-space solves of large patches in Gram form (subdomain size 4: 1176
// edges, 312 on the interface): a CTA takes PB patches at a time, gathers
// their residuals, forms t = W^t r_p (nG values per patch; threads along the
// columns of W, so W is read coalesced from L2) and y = W t (threads along
// the rows, reading W^t coalesced), and adds eta * y to z.
template <typename T, int PB>
__global__ void __launch_bounds__(256) k_patch_gram(int n, PatchFamily fam, int nG, const T* __restrict__ W,
                                                    const T* __restrict__ WT, T eta, const T* __restrict__ r,
                                                    T* __restrict__ z) {
  pdl_start();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nl = fam.nloc;
  T* Rs = reinterpret_cast<T*>(smem_raw);           // nl * PB
  T* Ts = Rs + (size_t)nl * PB;                      // nG * PB
  int* loc = reinterpret_cast<int*>(Ts + (size_t)nG * PB);
  const int64_t NP = (int64_t)fam.np[0] * fam.np[1] * fam.np[2];
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  r += (int64_t)blockIdx.y * 3 * N3;
  z += (int64_t)blockIdx.y * 3 * N3;
  const int bx = fam.b[0], by = fam.b[1], bz = fam.b[2];
  const int cx = bx * (by - 1) * (bz - 1), cy = (bx - 1) * by * (bz - 1);
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    int d, i, j, k, e = l;
    if (e < cx) {
      d = 0; i = e % bx; j = (e / bx) % (by - 1) + 1; k = e / (bx * (by - 1)) + 1;
    } else if ((e -= cx) < cy) {
      d = 1; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % by; k = e / ((bx - 1) * by) + 1;
    } else {
      e -= cy;
      d = 2; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % (by - 1) + 1; k = e / ((bx - 1) * (by - 1));
    }
    loc[l] = (((d * 16 + i) * 16 + j) * 16) + k;
  }
  auto gidx_of = [&](int64_t P, int l) {
    const int pa = (int)(P % fam.np[0]) + fam.p0[0];
    const int pb = (int)((P / fam.np[0]) % fam.np[1]) + fam.p0[1];
    const int pc = (int)(P / ((int64_t)fam.np[0] * fam.np[1])) + fam.p0[2];
    const int c = loc[l];
    const int d = c >> 12, i = (c >> 8) & 15, j = (c >> 4) & 15, k = c & 15;
    return edge_gidx(n, d, fam.stride * pa - fam.shift[0] + i, fam.stride * pb - fam.shift[1] + j,
                     fam.stride * pc - fam.shift[2] + k);
  };
  for (int64_t base = (int64_t)blockIdx.x * PB; base < NP; base += (int64_t)gridDim.x * PB) {
    __syncthreads();
    for (int q = threadIdx.x; q < nl * PB; q += blockDim.x) {
      const int p = q / nl, l = q % nl;
      const int64_t P = base + p;
      Rs[l * PB + p] = P < NP ? __ldg(r + gidx_of(P, l)) : T(0);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nG; c += blockDim.x) {
      T acc[PB];
#pragma unroll
      for (int p = 0; p < PB; ++p) acc[p] = T(0);
      for (int l = 0; l < nl; ++l) {
        const T w = __ldg(W + (size_t)l * nG + c);
#pragma unroll
        for (int p = 0; p < PB; ++p) acc[p] += w * Rs[l * PB + p];
      }
#pragma unroll
      for (int p = 0; p < PB; ++p) Ts[c * PB + p] = acc[p];
    }
    __syncthreads();
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
      T acc[PB];
#pragma unroll
      for (int p = 0; p < PB; ++p) acc[p] = T(0);
      for (int c = 0; c < nG; ++c) {
        const T w = __ldg(WT + (size_t)c * nl + l);
#pragma unroll
        for (int p = 0; p < PB; ++p) acc[p] += w * Ts[c * PB + p];
      }
#pragma unroll
      for (int p = 0; p < PB; ++p)
        if (base + p < NP) atomicAdd(z + gidx_of(base + p, l), eta * acc[p]);
    }
  }
}

// ---------------------------------------------------------------------------
// Local solves for a curl-curl coefficient that is constant per hexahedron.
// The local matrices of the subdomains (eq. ATDef) and patches (eq. AVDef,
// eq. AEDef) then depend on the coefficients of their cells; the host groups
// them by those values and builds one operator per group.
// ---------------------------------------------------------------------------
// Interior spaces: as k_bubble, with the 6x6 inverse of coarse element t at
// Atab + 36 gid[t] (coarse elements in x-fastest order).
template <typename T>
__global__ void __launch_bounds__(256) k_bubble_grouped(int n, const T* __restrict__ Atab, const int* __restrict__ gid,
                                                        T eta, const T* __restrict__ r, T* __restrict__ z) {
  pdl_start();
  const int nc = n / 2;
  const int64_t NT = (int64_t)nc * nc * nc;
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  r += (int64_t)blockIdx.y * 3 * N3;
  z += (int64_t)blockIdx.y * 3 * N3;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < NT; t += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(t % nc), J = (int)((t / nc) % nc), K = (int)(t / ((int64_t)nc * nc));
    const T* As = Atab + 36 * (int64_t)__ldg(gid + t);
    int64_t gi[6];
    int q = 0;
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        int p[3] = {2 * I + 1, 2 * J + 1, 2 * K + 1};
        p[d] = (d == 0 ? 2 * I : d == 1 ? 2 * J : 2 * K) + s;
        gi[q++] = edge_gidx(n, d, p[0], p[1], p[2]);
      }
    T rv[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) rv[a] = __ldg(r + gi[a]);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      T s = T(0);
#pragma unroll
      for (int b = 0; b < 6; ++b) s += __ldg(As + a * 6 + b) * rv[b];
      z[gi[a]] += eta * s;
    }
  }
}

// Patch solves with one dense operator per group: the patches of a family
// are listed group by group (plist), cut into chunks of at most PB patches of
// one group (chunk = {group, first list entry, count}); a CTA walks a
// contiguous range of chunks and stages a group's operator in shared memory
// only when the group changes.  z += eta * D_group r_p, atomics for overlaps.
template <typename T, int PB>
__global__ void __launch_bounds__(128) k_patch_grouped(int n, PatchFamily fam, const T* __restrict__ Dtab,
                                                       const int4* __restrict__ chunks, int nchunks,
                                                       const int* __restrict__ plist, T eta,
                                                       const T* __restrict__ r, T* __restrict__ z) {
  pdl_start();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nl = fam.nloc;
  T* Ds = reinterpret_cast<T*>(smem_raw);          // nl * nl
  T* Rs = Ds + nl * nl;                            // nl * PB
  int* loc = reinterpret_cast<int*>(Rs + nl * PB); // packed (d, i, j, k) of each local edge
  int* pidx = loc + nl;                            // PB patch numbers of the current chunk
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  r += (int64_t)blockIdx.y * 3 * N3;
  z += (int64_t)blockIdx.y * 3 * N3;
  const int bx = fam.b[0], by = fam.b[1], bz = fam.b[2];
  const int cx = bx * (by - 1) * (bz - 1), cy = (bx - 1) * by * (bz - 1);
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    int d, i, j, k, e = l;
    if (e < cx) {
      d = 0; i = e % bx; j = (e / bx) % (by - 1) + 1; k = e / (bx * (by - 1)) + 1;
    } else if ((e -= cx) < cy) {
      d = 1; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % by; k = e / ((bx - 1) * by) + 1;
    } else {
      e -= cy;
      d = 2; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % (by - 1) + 1; k = e / ((bx - 1) * (by - 1));
    }
    loc[l] = (((d * 16 + i) * 16 + j) * 16) + k;
  }
  auto gidx_of = [&](int64_t P, int l) {
    const int pa = (int)(P % fam.np[0]) + fam.p0[0];
    const int pb = (int)((P / fam.np[0]) % fam.np[1]) + fam.p0[1];
    const int pc = (int)(P / ((int64_t)fam.np[0] * fam.np[1])) + fam.p0[2];
    const int c = loc[l];
    const int d = c >> 12, i = (c >> 8) & 15, j = (c >> 4) & 15, k = c & 15;
    return edge_gidx(n, d, fam.stride * pa - fam.shift[0] + i, fam.stride * pb - fam.shift[1] + j,
                     fam.stride * pc - fam.shift[2] + k);
  };
  const int c0 = (int)((int64_t)blockIdx.x * nchunks / gridDim.x);
  const int c1 = (int)((int64_t)(blockIdx.x + 1) * nchunks / gridDim.x);
  int staged = -1;
  for (int ch = c0; ch < c1; ++ch) {
    const int4 cd = __ldg(chunks + ch);  // group, first entry, count
    __syncthreads();                     // the previous chunk is done with Ds, Rs, pidx
    if (cd.x != staged) {
      const T* D = Dtab + (int64_t)cd.x * nl * nl;
      for (int q = threadIdx.x; q < nl * nl; q += blockDim.x) Ds[q] = __ldg(D + q);
      staged = cd.x;
    }
    if (threadIdx.x < PB) pidx[threadIdx.x] = threadIdx.x < cd.z ? __ldg(plist + cd.y + threadIdx.x) : -1;
    __syncthreads();
    for (int q = threadIdx.x; q < nl * PB; q += blockDim.x) {
      const int p = q / nl, l = q % nl;
      const int P = pidx[p];
      Rs[l * PB + p] = P >= 0 ? __ldg(r + gidx_of(P, l)) : T(0);
    }
    __syncthreads();
    for (int row = threadIdx.x; row < nl; row += blockDim.x) {
      T acc[PB];
#pragma unroll
      for (int p = 0; p < PB; ++p) acc[p] = T(0);
      for (int c = 0; c < nl; ++c) {
        const T dv = Ds[c * nl + row];
#pragma unroll
        for (int p = 0; p < PB; ++p) acc[p] += dv * Rs[c * PB + p];
      }
#pragma unroll
      for (int p = 0; p < PB; ++p)
        if (pidx[p] >= 0) atomicAdd(z + gidx_of(pidx[p], row), eta * acc[p]);
    }
  }
}

// Per-hexahedron derivative of a(., .) in its coefficient: out_T = -lambda^T
// K_T u, K_T = h sum_d C_{T,d}^t m C_{T,d} (the curl of a lowest-order edge
// field on a cube has, per axis d, a component that varies linearly between
// the circulations of the two faces normal to d; m = [[1/3,1/6],[1/6,1/3]]).
// One thread per cell; out[rhs n^3 + (k n + j) n + i].
__device__ __forceinline__ double edge_val(const double* __restrict__ x, int n, int64_t N3, int d, int i, int j,
                                           int k) {
  if (d == 0) return in_seg(i, n) && in_node(j, n) && in_node(k, n) ? __ldg(x + off_x(n, i, j, k)) : 0.0;
  if (d == 1) return in_node(i, n) && in_seg(j, n) && in_node(k, n) ? __ldg(x + N3 + off_y(n, i, j, k)) : 0.0;
  return in_node(i, n) && in_node(j, n) && in_seg(k, n) ? __ldg(x + 2 * N3 + off_z(n, i, j, k)) : 0.0;
}

__device__ __forceinline__ void cell_circulations(const double* __restrict__ x, int n, int64_t N3, int i, int j,
                                                  int k, double c[3][2]) {
  double ex[2][2], ey[2][2], ez[2][2];  // x-edges [dj][dk], y-edges [di][dk], z-edges [di][dj]
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      ex[a][b] = edge_val(x, n, N3, 0, i, j + a, k + b);
      ey[a][b] = edge_val(x, n, N3, 1, i + a, j, k + b);
      ez[a][b] = edge_val(x, n, N3, 2, i + a, j + b, k);
    }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    c[0][s] = ez[s][1] - ez[s][0] - ey[s][1] + ey[s][0];  // x-normal face at x = i + s
    c[1][s] = ex[s][1] - ex[s][0] - ez[1][s] + ez[0][s];  // y-normal face at y = j + s
    c[2][s] = ey[1][s] - ey[0][s] - ex[1][s] + ex[0][s];  // z-normal face at z = k + s
  }
}

__global__ void __launch_bounds__(256) k_grad_cells(int n, double h, const double* __restrict__ lam,
                                                    const double* __restrict__ u, double* __restrict__ out) {
  pdl_start();
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  const int64_t NC = (int64_t)n * n * n;
  lam += (int64_t)blockIdx.y * 3 * N3;
  u += (int64_t)blockIdx.y * 3 * N3;
  out += (int64_t)blockIdx.y * NC;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < NC; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)((t / n) % n), k = (int)(t / ((int64_t)n * n));
    double a[3][2], b[3][2];
    cell_circulations(lam, n, N3, i, j, k, a);
    cell_circulations(u, n, N3, i, j, k, b);
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d)
      s += 2.0 * (a[d][0] * b[d][0] + a[d][1] * b[d][1]) + a[d][0] * b[d][1] + a[d][1] * b[d][0];
    out[t] = -h * s / 6.0;
  }
}

// ---------------------------------------------------------------------------
// Coarsest solve (Fig. 1, k = 0): z = A_0^{-1} g with the precomputed dense
// inverse (symmetric, so row i is column i): one warp per row, lanes along
// the row (coalesced), g staged in shared memory; 8 rows per CTA.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_coarse(int N0, const double* __restrict__ Ainv, const T* __restrict__ g,
                                                T* __restrict__ z) {
  pdl_start();
  extern __shared__ double gs[];
  g += (int64_t)blockIdx.y * N0;
  z += (int64_t)blockIdx.y * N0;
  for (int i = threadIdx.x; i < N0; i += blockDim.x) gs[i] = (double)g[i];
  __syncthreads();
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= N0) return;
  const double* a = Ainv + (int64_t)row * N0;
  double s = 0.0;
  for (int j = lane; j < N0; j += 32) s += __ldg(a + j) * gs[j];
  s = warp_sum(s);
  if (lane == 0) z[row] = (T)s;
}

// ---------------------------------------------------------------------------
// BLAS-1 with FP64 accumulation.  Reductions are two-stage and deterministic:
// a fixed number of blocks writes partial sums, one block adds them.
// ---------------------------------------------------------------------------

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

// Batched BLAS-1: grid y (or x for the finishing kernel) is the right-hand
// side; every right-hand side is a contiguous vector of N entries; scalars
// come from per-right-hand-side device arrays.
// partial[(rhs * gridDim.x + b) * 2 + {0,1}] = block sums of x.y and x2.y2
template <typename T>
__global__ void __launch_bounds__(256) k_dot2(int64_t N, const T* __restrict__ x, const T* __restrict__ y,
                                              const T* __restrict__ x2, const T* __restrict__ y2,
                                              double* __restrict__ partial) {
  pdl_start();
  const int64_t off = (int64_t)blockIdx.y * N;
  double v[2] = {0.0, 0.0};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    v[0] += (double)x[off + e] * (double)y[off + e];
    if (x2) v[1] += (double)x2[off + e] * (double)y2[off + e];
  }
  block_sum_store<2>(v, partial + 2 * ((int64_t)blockIdx.y * gridDim.x + blockIdx.x));
}

__global__ void k_finish2(int nb, const double* __restrict__ partial, double* __restrict__ out) {
  pdl_start();
  partial += 2 * (int64_t)blockIdx.x * nb;
  double v[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    v[0] += partial[2 * b];
    v[1] += partial[2 * b + 1];
  }
  block_sum_store<2>(v, out + 2 * blockIdx.x);
}

// dL/dalpha = -lambda^T K u in one pass: per cell the face pairs of the
// circulations of lambda and u (as k_grad_cells, times the cell's
// coefficient when acell is given, i.e. K = sum_T alpha_T K_T), accumulated
// in FP64 per thread and reduced per block into partial (layout of k_dot2,
// second slot 0); k_finish2 adds the blocks of every right-hand side
__global__ void __launch_bounds__(256) k_grad_alpha_sum(int n, double h, const double* __restrict__ lam,
                                                        const double* __restrict__ u,
                                                        const double* __restrict__ acell,
                                                        double* __restrict__ partial) {
  pdl_start();
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  const int64_t NC = (int64_t)n * n * n;
  lam += (int64_t)blockIdx.y * 3 * N3;
  u += (int64_t)blockIdx.y * 3 * N3;
  double v[2] = {0.0, 0.0};
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < NC; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)((t / n) % n), k = (int)(t / ((int64_t)n * n));
    double a[3][2], b[3][2];
    cell_circulations(lam, n, N3, i, j, k, a);
    cell_circulations(u, n, N3, i, j, k, b);
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d)
      s += 2.0 * (a[d][0] * b[d][0] + a[d][1] * b[d][1]) + a[d][0] * b[d][1] + a[d][1] * b[d][0];
    v[0] += acell ? acell[t] * s : s;
  }
  v[0] *= -h / 6.0;
  block_sum_store<2>(v, partial + 2 * ((int64_t)blockIdx.y * gridDim.x + blockIdx.x));
}

// PCG scalars kept on the device (one block per right-hand side, which
// first adds the block partial sums of one reduction in the layout of
// k_dot2): the host then reads one residual norm per iteration instead of
// three inner products.
//   CG_ALPHA: p.q -> alpha = rz / p.q (0 for a converged right-hand side;
//             a non-positive or non-finite curvature sets kStatusBreakdown);
//             also the scales sto = 2^-e, sfrom = 2^e of the last rr
//             (2^(e-1) <= ||r|| < 2^e)
//   CG_RR:    rr = r.r
//   CG_BETA:  r.z -> beta = rz_new / rz (textbook CG), rz = rz_new
//   CG_BETA_FLEX: r.z32, q.z32 with z = sfrom z32 -> beta = -alpha q.z / rz
//             (flexible form), rz = r.z
//   CG_RZ:    rz = scale r.z (scale = sfrom for a float preconditioner, else 1)
__global__ void k_cg_scalars(int mode, int nb, const double* __restrict__ partial, CgScalars S, int flex,
                             int* __restrict__ status) {
  pdl_start();
  partial += 2 * (int64_t)blockIdx.x * nb;
  double v[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    v[0] += partial[2 * b];
    v[1] += partial[2 * b + 1];
  }
  __shared__ double tot[2];
  block_sum_store<2>(v, tot);
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int i = blockIdx.x;
  const double s0 = tot[0], s1 = tot[1];
  const bool done = S.done[i] != 0.0;
  if (mode == CG_ALPHA) {
    double a = 0.0;
    if (!done) {
      if (s0 > 0.0 && isfinite(s0)) a = S.rz[i] / s0;
      else atomicOr(status, kStatusBreakdown);
    }
    S.alpha[i] = a;
    // the float V-cycle's input scale: sto = 2^-e, sfrom = 2^e with
    // 2^(e-1) <= ||r|| < 2^e, so that ||sto r|| lies in [1/2, 1) and both
    // scalings are exact exponent shifts (k_cg_update_rr, k_axpby_zf)
    const double rn = sqrt(S.rr[i]);
    if (rn > 0.0 && isfinite(rn)) {
      int e = ilogb(rn) + 1;
      e = e < -1022 ? -1022 : (e > 1022 ? 1022 : e);  // both scales stay normal doubles
      S.sto[i] = ldexp(1.0, -e);
      S.sfrom[i] = ldexp(1.0, e);
    } else {
      S.sto[i] = 0.0;
      S.sfrom[i] = rn;
    }
  } else if (mode == CG_RR) {
    S.rr[i] = s0;
  } else if (mode == CG_BETA || mode == CG_BETA_FLEX) {
    const double rz_new = mode == CG_BETA ? s0 : S.sfrom[i] * s0;
    double b = 0.0;
    if (!done && S.rz[i] != 0.0)
      b = mode == CG_BETA ? rz_new / S.rz[i] : -S.alpha[i] * (S.sfrom[i] * s1) / S.rz[i];
    S.rz[i] = rz_new;
    S.ab[2 * i] = 1.0;
    S.ab[2 * i + 1] = b;
  } else {  // CG_RZ
    S.rz[i] = (flex ? S.sfrom[i] : 1.0) * s0;
  }
}

// y = a x + b y with (a, b) = ab[2 rhs], ab[2 rhs + 1]
template <typename T>
__global__ void __launch_bounds__(256) k_axpby(int64_t N, const double* __restrict__ ab, const T* __restrict__ x,
                                               T* __restrict__ y) {
  pdl_start();
  const int64_t off = (int64_t)blockIdx.y * N;
  const double a = ab[2 * blockIdx.y], b = ab[2 * blockIdx.y + 1];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    y[off + e] = (T)(a * (double)x[off + e] + b * (double)y[off + e]);
}

// y = a x + b y with host scalars over a whole batch (y is not read when b = 0)
template <typename T>
__global__ void __launch_bounds__(256) k_axpby_scalar(int64_t N, double a, const T* __restrict__ x, double b,
                                                      T* __restrict__ y) {
  pdl_start();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = b == 0.0 ? (T)(a * (double)x[e]) : (T)(a * (double)x[e] + b * (double)y[e]);
}

// u += a p ; r -= a q with a = alpha[rhs]
template <typename T>
__global__ void __launch_bounds__(256) k_cg_update(int64_t N, const double* __restrict__ alpha, const T* __restrict__ p,
                                                   const T* __restrict__ q, T* __restrict__ u, T* __restrict__ r) {
  pdl_start();
  const int64_t off = (int64_t)blockIdx.y * N;
  const double a = alpha[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    u[off + e] = (T)((double)u[off + e] + a * (double)p[off + e]);
    r[off + e] = (T)((double)r[off + e] - a * (double)q[off + e]);
  }
}

// Fused steps of the mixed flexible PCG (FP64 vectors, float preconditioner):
// u += a p ; r -= a q ; g32 = sto * r (the float right-hand side of the next
// V-cycle) and block sums of r.r (partials in the layout of k_dot2).  sto is
// a power of two (k_cg_scalars), so g32 is the rounded r with its exponent
// shifted, formed on the integer pipe (d2f_pow2): three FP64 operations per
// entry instead of five
__global__ void __launch_bounds__(256) k_cg_update_rr(int64_t N, const double* __restrict__ alpha,
                                                      const double* __restrict__ p, const double* __restrict__ q,
                                                      double* __restrict__ u, double* __restrict__ r,
                                                      const double* __restrict__ sto, float* __restrict__ g32,
                                                      double* __restrict__ partial) {
  pdl_start();
  const int64_t off = (int64_t)blockIdx.y * N;
  const double a = alpha[blockIdx.y];
  const int ks = pow2_exponent(sto[blockIdx.y]);
  double v[2] = {0.0, 0.0};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    u[off + e] += a * p[off + e];
    const double rn = r[off + e] - a * q[off + e];
    r[off + e] = rn;
    g32[off + e] = d2f_pow2(rn, ks);
    v[0] += rn * rn;
  }
  block_sum_store<2>(v, partial + 2 * ((int64_t)blockIdx.y * gridDim.x + blockIdx.x));
}

// block sums of x.z32 and y.z32 (the preconditioned residual is sc * z32;
// the caller applies sc to the two sums, one FP64 product per sum instead of
// one per entry)
// umax0 (optional): the next stencil's max |p| words, set to 0 here for
// k_axpby_zf to fill
__global__ void __launch_bounds__(256) k_dot2_zf(int64_t N, const double* __restrict__ x, const double* __restrict__ y,
                                                 const float* __restrict__ z32, double* __restrict__ partial,
                                                 unsigned long long* __restrict__ umax0) {
  pdl_start();
  if (umax0 && blockIdx.x == 0 && threadIdx.x == 0) umax0[blockIdx.y] = 0ull;
  const int64_t off = (int64_t)blockIdx.y * N;
  double v[2] = {0.0, 0.0};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const double z = f2d_bits(z32[off + e]);
    v[0] += x[off + e] * z;
    v[1] += y[off + e] * z;
  }
  block_sum_store<2>(v, partial + 2 * ((int64_t)blockIdx.y * gridDim.x + blockIdx.x));
}

// p = sc * z32 + b p with b = ab[2 rhs + 1]; sc is a power of two
// (k_cg_scalars), so sc * z32 is exact and formed on the integer pipe
// (f2d_pow2), one FP64 operation per entry; umax (optional, 0 on entry):
// max |p| of each right-hand side as k_absmax forms it, for the fixed-point
// stencil that applies A to p next
__global__ void __launch_bounds__(256) k_axpby_zf(int64_t N, const double* __restrict__ sc, const float* __restrict__ z32,
                                                  const double* __restrict__ ab, double* __restrict__ p,
                                                  unsigned long long* __restrict__ umax) {
  pdl_start();
  const int64_t off = (int64_t)blockIdx.y * N;
  const int ks = pow2_exponent(sc[blockIdx.y]);
  const double b = ab[2 * blockIdx.y + 1];
  unsigned long long m = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = fma(b, p[off + e], f2d_pow2(z32[off + e], ks));
    p[off + e] = v;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    m = bits > m ? bits : m;
  }
  if (umax) {  // one atomic per block (all blocks meet on one word per right-hand side)
    __shared__ unsigned long long wm[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
      m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = wm[w] > m ? wm[w] : m;
      if (m > 0) atomicMax(umax + blockIdx.y, m);
    }
  }
}

// dst (float) = s * src (double), s = sc[rhs]
__global__ void __launch_bounds__(256) k_to_f32(int64_t N, const double* __restrict__ sc, const double* __restrict__ src,
                                                float* __restrict__ dst) {
  pdl_start();
  const int64_t off = (int64_t)blockIdx.y * N;
  const double s = sc[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    dst[off + e] = (float)(s * src[off + e]);
}

// dst (double) = s * src (float)
__global__ void __launch_bounds__(256) k_from_f32(int64_t N, const double* __restrict__ sc, const float* __restrict__ src,
                                                  double* __restrict__ dst) {
  pdl_start();
  const int64_t off = (int64_t)blockIdx.y * N;
  const double s = sc[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    dst[off + e] = s * (double)src[off + e];
}

// dst (double) += s * src (float)
__global__ void __launch_bounds__(256) k_add_f32(int64_t N, const double* __restrict__ sc, const float* __restrict__ src,
                                                 double* __restrict__ dst) {
  pdl_start();
  const int64_t off = (int64_t)blockIdx.y * N;
  const double s = sc[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    dst[off + e] += s * (double)src[off + e];
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
size_t stencil_smem() { return sizeof(T) * (15 * kP + 9 * kTP); }

// the FP64 operator runs in fixed point (k_stencil_stream<double, long long>)
template <typename T>
using StencilArith = typename std::conditional<std::is_same<T, double>::value, long long, T>::type;

template <typename T>
cudaError_t prepare_stencil() {
  return cudaFuncSetAttribute(k_stencil_stream<T, StencilArith<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)stencil_smem<T>());
}

// z chunk: the longest (fewest halo planes) that still gives about four
// CTAs per SM
// (kz > 0: the chunk length chosen by ndmg_autotune)
static inline dim3 stencil_grid(int n, int sm, int R, int* KZ, int kz_choice) {
  const int64_t cols = (int64_t)((n + kTX - 1) / kTX) * ((n + kTY - 1) / kTY) * R;
  int kz = n;
  while (kz > 2 && cols * ((n + kz - 1) / kz) < 4LL * sm) kz = (kz + 1) / 2;
  if (kz_choice > 0) kz = kz_choice < n ? kz_choice : n;
  *KZ = kz;
  return dim3((n + kTX - 1) / kTX, (n + kTY - 1) / kTY, ((n + kz - 1) / kz) * R);
}

template <typename T>
int launch_stencil(cudaStream_t s, int sm, int n, double cK, double cM, const T* u, const T* g, T* y, int R,
                   unsigned long long* umax, int kz, bool umax_ready, double* pq, int64_t pq_cap) {
  const int64_t N = 3LL * n * (n - 1) * (n - 1);
  if (N == 0) return 0;
  if constexpr (std::is_same<T, double>::value) if (!umax_ready) {
    cudaMemsetAsync(umax, 0, sizeof(unsigned long long) * R, s);
    launch_pdl(k_absmax, dim3(grid_for(N, sm, 4), R), 256, 0, s, N, u, umax);
  }
  int KZ = 0;
  const dim3 grid = stencil_grid(n, sm, R, &KZ, kz);
  // the fused curvature sums: the fixed-point apply only, and only when the
  // blocks of one right-hand side fit the caller's buffer
  const int64_t nb = (int64_t)grid.x * grid.y * (grid.z / R);
  const bool fuse = std::is_same<T, double>::value && g == nullptr && pq != nullptr && nb <= pq_cap;
  launch_pdl(k_stencil_stream<T, StencilArith<T>>, grid, dim3(kTX, kTY), stencil_smem<T>(), s, n, KZ, (T)cK, (T)cM, u, g,
             y, (const unsigned long long*)umax, (const T*)nullptr, fuse ? pq : (double*)nullptr);
  return fuse ? (int)nb : 0;
}

// coefficient field: three more staged planes (the cell coefficients)
template <typename T>
size_t stencil_field_smem() { return stencil_smem<T>() + sizeof(T) * 4 * kP; }

template <typename T>
cudaError_t prepare_stencil_field() {
  return cudaFuncSetAttribute(k_stencil_stream<T, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)stencil_field_smem<T>());
}

template <typename T>
void launch_stencil_field(cudaStream_t s, int sm, int n, double cK, double cM, const T* u, const T* g, T* y, int R,
                          const T* acell, int kz) {
  if (n < 2) return;
  int KZ = 0;
  const dim3 grid = stencil_grid(n, sm, R, &KZ, kz);
  launch_pdl(k_stencil_stream<T, T, true>, grid, dim3(kTX, kTY), stencil_field_smem<T>(), s, n, KZ, (T)cK, (T)cM, u, g, y, nullptr, acell,
             (double*)nullptr);
}

// grid z of the transfers = coarse planes x right-hand sides; batches whose
// product would pass the 65,535 limit of grid z go in groups of right-hand
// sides (contiguous vectors, so a group is a pointer offset)
constexpr int kMaxGridZ = 65535;
// fine grids from this size on take the per-coarse-cell prolongation kernel
constexpr int kProlongCellMinN = 128;

template <typename T>
void launch_restrict(cudaStream_t s, int, int nf, const T* rf, T* gc, int R, T* zc) {
  const int nc = nf / 2;
  if (nc < 2) return;
  const int64_t Nf = 3LL * nf * (nf - 1) * (nf - 1), Nc = 3LL * nc * (nc - 1) * (nc - 1);
  const int group = kMaxGridZ / nc;
  for (int r0 = 0; r0 < R; r0 += group) {
    const int rg = R - r0 < group ? R - r0 : group;
    launch_pdl(k_restrict<T>, dim3((nc + 31) / 32, (nc + 7) / 8, nc * rg), dim3(32, 8), 0, s, nf, rf + r0 * Nf, gc + r0 * Nc,
               zc ? zc + r0 * Nc : zc);
  }
}

template <typename T>
void launch_prolong_add(cudaStream_t s, int, int nf, const T* zc, T* zf, int R) {
  const int nc = nf / 2;
  if (nc < 1) return;
  const int64_t Nf = 3LL * nf * (nf - 1) * (nf - 1), Nc = 3LL * nc * (nc - 1) * (nc - 1);
  if (nf >= kProlongCellMinN) {
    const int group = kMaxGridZ / nc;
    for (int r0 = 0; r0 < R; r0 += group) {
      const int rg = R - r0 < group ? R - r0 : group;
      launch_pdl(k_prolong_add_cell<T>, dim3((nc + 31) / 32, (nc + 7) / 8, nc * rg), dim3(32, 8), 0, s, nf,
                 zc + r0 * Nc, zf + r0 * Nf);
    }
    return;
  }
  const int group = kMaxGridZ / nf;
  for (int r0 = 0; r0 < R; r0 += group) {
    const int rg = R - r0 < group ? R - r0 : group;
    launch_pdl(k_prolong_add<T>, dim3((nf + 31) / 32, (nf + 7) / 8, nf * rg), dim3(32, 8), 0, s, nf, zc + r0 * Nc,
                                                                                          zf + r0 * Nf);
  }
}

template <typename T>
void launch_bubble(cudaStream_t s, int sm, int n, const T* Ainv, double eta, const T* r, T* z, int R) {
  const int64_t nc = n / 2;
  launch_pdl(k_bubble<T>, dim3(grid_for(nc * nc * nc, sm, 16), R), 256, 0, s, n, Ainv, (T)eta, r, z);
}

constexpr int kPB64 = 8;
constexpr int kPB32 = 16;

template <typename T>
static constexpr int pb_for() { return sizeof(T) == 8 ? kPB64 : kPB32; }

template <typename T>
size_t patch_dense_smem(int nloc) { return sizeof(T) * (nloc * nloc + nloc * pb_for<T>()) + sizeof(int) * nloc; }

// double-float kernel for FP64 vectors: hi / lo floats of D and of the
// pass's residuals, local offsets, patch origins, the pass maximum
size_t patch_dense_df_smem(int nloc) {
  return sizeof(float) * 2 * ((size_t)((nloc * nloc + 3) & ~3) + (size_t)nloc * kPBdf) +
         sizeof(int) * ((nloc + 1) & ~1) + sizeof(long long) * 3 * kPBdf + 16;
}

template <typename T>
cudaError_t prepare_vertex_dense() {
  if constexpr (std::is_same<T, double>::value)
    return cudaFuncSetAttribute(k_patch_dense_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)patch_dense_df_smem(108));
  else
    return cudaFuncSetAttribute(k_patch_dense<T, pb_for<T>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)patch_dense_smem<T>(108));
}

template <typename T>
void launch_patch_dense(cudaStream_t s, int sm, int n, const PatchFamily& fam, const T* D, double eta, const T* r,
                        T* z, int R) {
  const int64_t NP = (int64_t)fam.np[0] * fam.np[1] * fam.np[2];
  if (NP <= 0) return;
  constexpr int PB = pb_for<T>();
  int64_t blocks = (NP + PB - 1) / PB;
  const int64_t cap = (int64_t)sm * 2;
  if (blocks > cap) blocks = cap;
  if constexpr (std::is_same<T, double>::value) {
    int64_t bdf = (NP + kPBdf - 1) / kPBdf;
    if (bdf > cap) bdf = cap;
    launch_pdl(k_patch_dense_df, dim3((int)bdf, R), kDfThreads, patch_dense_df_smem(fam.nloc), s, n, fam, D, eta, r,
               z);
  } else {
    launch_pdl(k_patch_dense<T, PB>, dim3((int)blocks, R), 128, patch_dense_smem<T>(fam.nloc), s, n, fam, D, (T)eta,
               r, z);
  }
}

// levels with at most this many vertex patches take k_smooth_direct
constexpr int64_t kDirectMaxPatches = 4096;
constexpr int kPBdirect = 4;

bool smooth_direct_fits(int n) {
  const int64_t nv = n / 2 - 1;
  return nv >= 1 && nv * nv * nv <= kDirectMaxPatches;
}

void launch_smooth_direct(cudaStream_t s, int n, const float* D, const float* Ainv, double eta, const float* r,
                          float* z, int R) {
  const PatchFamily fam = vertex_family(n);
  const int64_t NP = (int64_t)fam.np[0] * fam.np[1] * fam.np[2];
  const int64_t nc = n / 2;
  const int npb = (int)((NP + kPBdirect - 1) / kPBdirect);
  const int nbb = (int)((nc * nc * nc + 127) / 128);
  launch_pdl(k_smooth_direct<kPBdirect>, dim3(npb + nbb, R), 128, sizeof(float) * 108 * 108, s, n, fam, D, Ainv,
             (float)eta, npb, r, z);
}

cudaError_t prepare_smooth_direct() {
  return cudaFuncSetAttribute(k_smooth_direct<kPBdirect>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(float) * 108 * 108));
}

PatchFamily vertex_family(int n) {
  const int nv = n / 2 - 1;
  return PatchFamily{108, {4, 4, 4}, {nv, nv, nv}, {1, 1, 1}, {2, 2, 2}};
}

PatchFamily subdomain4_family(int n) {
  const int nc = n / 4;
  PatchFamily f{108, {4, 4, 4}, {nc, nc, nc}, {0, 0, 0}, {0, 0, 0}};
  f.stride = 4;
  return f;
}

PatchFamily vertex4_family(int n) {
  const int nv = n / 4 - 1;
  PatchFamily f{1176, {8, 8, 8}, {nv, nv, nv}, {1, 1, 1}, {4, 4, 4}};
  f.stride = 4;
  return f;
}

constexpr int kGramPB64 = 8, kGramPB32 = 16;
template <typename T>
static constexpr int gram_pb() { return sizeof(T) == 8 ? kGramPB64 : kGramPB32; }
template <typename T>
size_t patch_gram_smem(int nloc, int nG) {
  return sizeof(T) * (size_t)(nloc + nG) * gram_pb<T>() + sizeof(int) * nloc;
}

template <typename T>
cudaError_t prepare_patch_gram() {
  return cudaFuncSetAttribute(k_patch_gram<T, gram_pb<T>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)patch_gram_smem<T>(1176, 312));
}

template <typename T>
void launch_patch_gram(cudaStream_t s, int sm, int n, const PatchFamily& fam, int nG, const T* W, const T* WT,
                       double eta, const T* r, T* z, int R) {
  const int64_t NP = (int64_t)fam.np[0] * fam.np[1] * fam.np[2];
  if (NP <= 0) return;
  constexpr int PB = gram_pb<T>();
  int64_t blocks = (NP + PB - 1) / PB;
  const int64_t cap = (int64_t)sm * 2;
  if (blocks > cap) blocks = cap;
  launch_pdl(k_patch_gram<T, PB>, dim3((int)blocks, R), 256, patch_gram_smem<T>(fam.nloc, nG), s, n, fam, nG, W, WT,
                                                                                           (T)eta, r, z);
}

PatchFamily edge_family(int n, int d) {
  const int nc = n / 2;
  PatchFamily f{42, {4, 4, 4}, {nc - 1, nc - 1, nc - 1}, {1, 1, 1}, {2, 2, 2}};
  f.b[d] = 2;
  f.np[d] = nc;
  f.p0[d] = 0;
  f.shift[d] = 0;
  return f;
}

template <typename T>
void launch_vertex_dense(cudaStream_t s, int sm, int n, const T* D, double eta, const T* r, T* z, int R) {
  launch_patch_dense<T>(s, sm, n, vertex_family(n), D, eta, r, z, R);
}

template <typename T>
void launch_coarse(cudaStream_t s, int N0, const double* Ainv, const T* g, T* z, int R) {
  launch_pdl(k_coarse<T>, dim3((N0 + 7) / 8, R), 256, sizeof(double) * N0, s, N0, Ainv, g, z);
}

int reduction_blocks(int sm) { return sm * 4; }

template <typename T>
void launch_dot2(cudaStream_t s, int sm, int64_t N, const T* x, const T* y, const T* x2, const T* y2, double* partial,
                 double* out, int R) {
  const int nb = reduction_blocks(sm);
  launch_pdl(k_dot2<T>, dim3(nb, R), 256, 0, s, N, x, y, x2, y2, partial);
  launch_pdl(k_finish2, R, 256, 0, s, nb, partial, out);
}

template <typename T>
void launch_dot2_partial(cudaStream_t s, int sm, int64_t N, const T* x, const T* y, const T* x2, const T* y2,
                         double* partial, int R) {
  launch_pdl(k_dot2<T>, dim3(reduction_blocks(sm), R), 256, 0, s, N, x, y, x2, y2, partial);
}
template void launch_dot2_partial<double>(cudaStream_t, int, int64_t, const double*, const double*, const double*,
                                          const double*, double*, int);

void launch_cg_update_rr_partial(cudaStream_t s, int sm, int64_t N, const double* alpha, const double* p,
                                 const double* q, double* u, double* r, const double* sto, float* g32,
                                 double* partial, int R) {
  launch_pdl(k_cg_update_rr, dim3(reduction_blocks(sm), R), 256, 0, s, N, alpha, p, q, u, r, sto, g32, partial);
}
void launch_dot2_zf_partial(cudaStream_t s, int sm, int64_t N, const double* x, const double* y, const float* z32,
                            double* partial, int R, unsigned long long* umax0) {
  launch_pdl(k_dot2_zf, dim3(reduction_blocks(sm), R), 256, 0, s, N, x, y, z32, partial, umax0);
}

static inline dim3 blas_grid(int64_t N, int sm, int R) {
  const int per = R > 1 ? 2 : 8;
  return dim3(grid_for(N, sm, per), R);
}

template <typename T>
void launch_axpby(cudaStream_t s, int sm, int64_t N, const double* ab, const T* x, T* y, int R) {
  launch_pdl(k_axpby<T>, blas_grid(N, sm, R), 256, 0, s, N, ab, x, y);
}

template <typename T>
void launch_axpby_scalar(cudaStream_t s, int sm, int64_t N, double a, const T* x, double b, T* y) {
  if (N <= 0) return;
  launch_pdl(k_axpby_scalar<T>, grid_for(N, sm, 8), 256, 0, s, N, a, x, b, y);
}

template <typename T>
void launch_cg_update(cudaStream_t s, int sm, int64_t N, const double* alpha, const T* p, const T* q, T* u, T* r, int R) {
  launch_pdl(k_cg_update<T>, blas_grid(N, sm, R), 256, 0, s, N, alpha, p, q, u, r);
}

void launch_cg_update_rr(cudaStream_t s, int sm, int64_t N, const double* alpha, const double* p, const double* q,
                         double* u, double* r, const double* sto, float* g32, double* partial, double* out, int R) {
  const int nb = reduction_blocks(sm);
  launch_pdl(k_cg_update_rr, dim3(nb, R), 256, 0, s, N, alpha, p, q, u, r, sto, g32, partial);
  launch_pdl(k_finish2, R, 256, 0, s, nb, partial, out);
}
void launch_dot2_zf(cudaStream_t s, int sm, int64_t N, const double* x, const double* y, const float* z32,
                    double* partial, double* out, int R) {
  const int nb = reduction_blocks(sm);
  launch_pdl(k_dot2_zf, dim3(nb, R), 256, 0, s, N, x, y, z32, partial, (unsigned long long*)nullptr);
  launch_pdl(k_finish2, R, 256, 0, s, nb, partial, out);
}
void launch_axpby_zf(cudaStream_t s, int sm, int64_t N, const double* sc, const float* z32, const double* ab, double* p,
                     int R, unsigned long long* umax) {
  launch_pdl(k_axpby_zf, blas_grid(N, sm, R), 256, 0, s, N, sc, z32, ab, p, umax);
}

void launch_to_f32(cudaStream_t s, int sm, int64_t N, const double* sc, const double* src, float* dst, int R) {
  launch_pdl(k_to_f32, blas_grid(N, sm, R), 256, 0, s, N, sc, src, dst);
}
void launch_from_f32(cudaStream_t s, int sm, int64_t N, const double* sc, const float* src, double* dst, int R) {
  launch_pdl(k_from_f32, blas_grid(N, sm, R), 256, 0, s, N, sc, src, dst);
}
void launch_add_f32(cudaStream_t s, int sm, int64_t N, const double* sc, const float* src, double* dst, int R) {
  launch_pdl(k_add_f32, blas_grid(N, sm, R), 256, 0, s, N, sc, src, dst);
}

// ---- coefficient field ------------------------------------------------------
template <typename T>
void launch_bubble_grouped(cudaStream_t s, int sm, int n, const T* Atab, const int* gid, double eta, const T* r, T* z,
                           int R) {
  const int64_t nc = n / 2;
  launch_pdl(k_bubble_grouped<T>, dim3(grid_for(nc * nc * nc, sm, 16), R), 256, 0, s, n, Atab, gid, (T)eta, r, z);
}

constexpr int kGroupPB = 8;

template <typename T>
size_t patch_grouped_smem(int nloc) {
  return sizeof(T) * (size_t)(nloc * nloc + nloc * kGroupPB) + sizeof(int) * (size_t)(nloc + kGroupPB);
}

template <typename T>
cudaError_t prepare_patch_grouped() {
  return cudaFuncSetAttribute(k_patch_grouped<T, kGroupPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)patch_grouped_smem<T>(108));
}

int patch_group_size() { return kGroupPB; }

template <typename T>
void launch_patch_grouped(cudaStream_t s, int sm, int n, const PatchFamily& fam, const T* Dtab, const int4* chunks,
                          int nchunks, const int* plist, double eta, const T* r, T* z, int R) {
  if (nchunks <= 0) return;
  int blocks = sm * 2;
  if (blocks > nchunks) blocks = nchunks;
  launch_pdl(k_patch_grouped<T, kGroupPB>, dim3(blocks, R), 128, patch_grouped_smem<T>(fam.nloc), s, 
      n, fam, Dtab, chunks, nchunks, plist, (T)eta, r, z);
}

void launch_cg_scalars(cudaStream_t s, int mode, int nb, const double* partial, const CgScalars& S, bool flex,
                       int* status, int R) {
  launch_pdl(k_cg_scalars, R, 256, 0, s, mode, nb, partial, S, flex ? 1 : 0, status);
}

void launch_grad_alpha_sum(cudaStream_t s, int sm, int n, double h, const double* lam, const double* u,
                           const double* acell, double* partial, double* out, int R) {
  const int nb = reduction_blocks(sm);
  launch_pdl(k_grad_alpha_sum, dim3(nb, R), 256, 0, s, n, h, lam, u, acell, partial);
  launch_pdl(k_finish2, R, 256, 0, s, nb, partial, out);
}

void launch_grad_cells(cudaStream_t s, int sm, int n, double h, const double* lam, const double* u, double* out,
                       int R) {
  const int64_t nc = (int64_t)n * n * n;
  launch_pdl(k_grad_cells, dim3(grid_for(nc, sm, 8), R), 256, 0, s, n, h, lam, u, out);
}

#define NDMG_INST(T)                                                                                   \
  template int launch_stencil<T>(cudaStream_t, int, int, double, double, const T*, const T*, T*, int,     \
                                 unsigned long long*, int, bool, double*, int64_t);                   \
  template cudaError_t prepare_stencil<T>();                                                          \
  template cudaError_t prepare_stencil_field<T>();                                                    \
  template void launch_stencil_field<T>(cudaStream_t, int, int, double, double, const T*, const T*, T*, int, \
                                        const T*, int);                                               \
  template void launch_bubble_grouped<T>(cudaStream_t, int, int, const T*, const int*, double, const T*, T*, int); \
  template cudaError_t prepare_patch_grouped<T>();                                                    \
  template void launch_patch_grouped<T>(cudaStream_t, int, int, const PatchFamily&, const T*, const int4*, int, \
                                        const int*, double, const T*, T*, int);                       \
  template void launch_restrict<T>(cudaStream_t, int, int, const T*, T*, int, T*);                    \
  template void launch_prolong_add<T>(cudaStream_t, int, int, const T*, T*, int);                     \
  template void launch_bubble<T>(cudaStream_t, int, int, const T*, double, const T*, T*, int);        \
  template cudaError_t prepare_vertex_dense<T>();                                                     \
  template void launch_vertex_dense<T>(cudaStream_t, int, int, const T*, double, const T*, T*, int);  \
  template void launch_patch_dense<T>(cudaStream_t, int, int, const PatchFamily&, const T*, double, const T*, T*, int); \
  template void launch_coarse<T>(cudaStream_t, int, const double*, const T*, T*, int);                \
  template void launch_dot2<T>(cudaStream_t, int, int64_t, const T*, const T*, const T*, const T*,    \
                               double*, double*, int);                                                \
  template void launch_axpby<T>(cudaStream_t, int, int64_t, const double*, const T*, T*, int);         \
  template void launch_patch_gram<T>(cudaStream_t, int, int, const PatchFamily&, int, const T*, const T*, \
                                     double, const T*, T*, int);                                       \
  template cudaError_t prepare_patch_gram<T>();                                                       \
  template void launch_axpby_scalar<T>(cudaStream_t, int, int64_t, double, const T*, double, T*);      \
  template void launch_cg_update<T>(cudaStream_t, int, int64_t, const double*, const T*, const T*, T*, T*, int);
NDMG_INST(double)
NDMG_INST(float)

}  // namespace ndmg
