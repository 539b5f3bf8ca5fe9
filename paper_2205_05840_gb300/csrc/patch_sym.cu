// FP64 dense patch solves z += eta * D r_p (eq. (Preconditioner P): the
// vertex-space operator J_V A_V^{-1} J_V^t; eq. (Preconditioner E): the
// edge-space ones) in a basis adapted to the patch's mirror symmetries.
//
// With a constant coefficient on a uniform grid a patch box is mapped onto
// itself by the three reflections through its centre, x -> b_x - x and so on
// (an edge along the reflected axis reverses its orientation, so its degree
// of freedom changes sign), and its matrix commutes with all three.  So does
// D.  The reflections generate the group Z2^3; its eight characters chi split
// the patch space into eigenspaces that D maps into themselves.  Each row of
// the transform T is the signed sum of the degrees of freedom of one edge
// orbit under the group for one character compatible with the orbit (entries
// +-1, rows orthogonal, T T^t = Lambda = the orbit sizes).  Then
//     D = T^t M T,   M = Lambda^{-1} (T D T^t) Lambda^{-1},
// and M is block diagonal, one block per character: for the 108-edge vertex
// patch the blocks have 24, 16, 16, 16, 10, 10, 10 and 6 rows, 1,680 entries
// against 11,664 for D, so the product costs a seventh of the dense one.
//
// The kernel keeps FP64 accuracy on the FP32 pipe: the residuals of a pass of
// patches are scaled by a power of two and taken to int64 fixed point, T is
// applied exactly in integers, each transformed entry becomes a pair of
// floats (48 significant bits), the block products run in double-float
// arithmetic (an exact product error by fma, error-free two-sums), T^t sums
// the block outputs the same way, and only the final value and its atomic
// addition into z are FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <vector>

#include "kernels.cuh"
#include "pdl.cuh"

namespace ndmg {

namespace {

// blob layout (32-bit words): [0] nloc, [1] blocks, [2] M entries;
// [3 + 3q ..] per block: first row, rows, offset of its entries in M;
// rows: 3 words each (members 0-3 and 4-7 as bytes, then count | signs << 8 |
// block << 16); edges: 3 words each (rows 0-3, 4-7, count | signs << 8);
// then M hi, M lo (floats, column-major per block)
constexpr int kHdr = 3 + 3 * 8;
__host__ __device__ constexpr int rows_at() { return kHdr; }
__host__ __device__ constexpr int edges_at(int nl) { return kHdr + 3 * nl; }
__host__ __device__ constexpr int m_at(int nl) { return kHdr + 6 * nl; }

struct Edge {
  int d, i, j, k;
};

// patch-local edge l of a box of b[0] x b[1] x b[2] cells (interior edges,
// the order every dense patch kernel uses)
Edge local_edge(const int b[3], int l) {
  const int bx = b[0], by = b[1], bz = b[2];
  const int cx = bx * (by - 1) * (bz - 1), cy = (bx - 1) * by * (bz - 1);
  Edge e;
  int q = l;
  if (q < cx) {
    e = {0, q % bx, (q / bx) % (by - 1) + 1, q / (bx * (by - 1)) + 1};
  } else if ((q -= cx) < cy) {
    e = {1, q % (bx - 1) + 1, (q / (bx - 1)) % by, q / ((bx - 1) * by) + 1};
  } else {
    q -= cy;
    e = {2, q % (bx - 1) + 1, (q / (bx - 1)) % (by - 1) + 1, q / ((bx - 1) * (by - 1))};
  }
  return e;
}

int local_index(const int b[3], const Edge& e) {
  const int bx = b[0], by = b[1], bz = b[2];
  const int cx = bx * (by - 1) * (bz - 1), cy = (bx - 1) * by * (bz - 1);
  if (e.d == 0) return e.i + bx * ((e.j - 1) + (by - 1) * (e.k - 1));
  if (e.d == 1) return cx + (e.i - 1) + (bx - 1) * (e.j + by * (e.k - 1));
  return cx + cy + (e.i - 1) + (bx - 1) * ((e.j - 1) + (by - 1) * e.k);
}

}  // namespace

bool build_patch_sym(const PatchFamily& fam, const double* D, std::vector<uint32_t>* blob, double* dropped) {
  const int nl = fam.nloc;
  if (nl > 128) return false;
  const int* b = fam.b;
  for (int l = 0; l < nl; ++l)
    if (local_index(b, local_edge(b, l)) != l) throw std::logic_error("patch-local edge numbering");
  // the image and sign of edge l under the group element g (bit a: reflect axis a)
  auto act = [&](int l, int g, int* sign) {
    Edge e = local_edge(b, l);
    int s = 1;
    int c[3] = {e.i, e.j, e.k};
    for (int a = 0; a < 3; ++a)
      if ((g >> a) & 1) {
        if (e.d == a) {
          c[a] = b[a] - 1 - c[a];
          s = -s;
        } else {
          c[a] = b[a] - c[a];
        }
      }
    *sign = s;
    return local_index(b, Edge{e.d, c[0], c[1], c[2]});
  };
  // rows: (character, orbit) pairs compatible with the orbit's stabiliser
  struct Row {
    int chi;
    std::vector<int> mem, sgn;
  };
  std::vector<Row> rows;
  for (int chi = 0; chi < 8; ++chi) {
    std::vector<bool> seen(nl, false);
    for (int l = 0; l < nl; ++l) {
      if (seen[l]) continue;
      // coefficient of each orbit member: chi(g) sign(g); compatible iff consistent
      std::vector<int> coef(nl, 0);
      bool ok = true;
      for (int g = 0; g < 8; ++g) {
        int s;
        const int m = act(l, g, &s);
        seen[m] = true;
        const int c = s * ((__builtin_popcount(g & chi) & 1) ? -1 : 1);
        if (coef[m] == 0) coef[m] = c;
        else if (coef[m] != c) ok = false;
      }
      if (!ok) continue;
      Row r{chi, {}, {}};
      for (int m = 0; m < nl; ++m)
        if (coef[m] != 0) {
          r.mem.push_back(m);
          r.sgn.push_back(coef[m]);
        }
      rows.push_back(r);
    }
  }
  if ((int)rows.size() != nl) return false;
  // block structure (rows are grouped by character by construction)
  std::vector<int> first, size;
  for (int r = 0; r < nl; ++r) {
    if (r == 0 || rows[r].chi != rows[r - 1].chi) {
      first.push_back(r);
      size.push_back(0);
    }
    ++size.back();
  }
  const int nb = (int)first.size();
  // Bt = T D T^t, M = Lambda^{-1} Bt Lambda^{-1} on the diagonal blocks
  std::vector<double> TD((size_t)nl * nl, 0.0);
  for (int r = 0; r < nl; ++r)
    for (size_t q = 0; q < rows[r].mem.size(); ++q) {
      const int m = rows[r].mem[q];
      for (int c = 0; c < nl; ++c) TD[(size_t)r * nl + c] += rows[r].sgn[q] * D[(size_t)m * nl + c];
    }
  std::vector<double> Bt((size_t)nl * nl, 0.0);
  for (int r = 0; r < nl; ++r)
    for (int s = 0; s < nl; ++s) {
      double v = 0.0;
      for (size_t q = 0; q < rows[s].mem.size(); ++q) v += TD[(size_t)r * nl + rows[s].mem[q]] * rows[s].sgn[q];
      Bt[(size_t)r * nl + s] = v;
    }
  double off = 0.0, all = 0.0;
  std::vector<int> blk(nl);
  for (int q = 0; q < nb; ++q)
    for (int r = first[q]; r < first[q] + size[q]; ++r) blk[r] = q;
  for (int r = 0; r < nl; ++r)
    for (int s = 0; s < nl; ++s) {
      const double v = Bt[(size_t)r * nl + s] / ((double)rows[r].mem.size() * rows[s].mem.size());
      all = std::max(all, std::fabs(v));
      if (blk[r] != blk[s]) off = std::max(off, std::fabs(v));
    }
  *dropped = all > 0 ? off / all : 0.0;
  int mtot = 0;
  for (int q = 0; q < nb; ++q) mtot += size[q] * size[q];
  blob->assign(m_at(nl) + 2 * mtot, 0u);
  uint32_t* w = blob->data();
  w[0] = nl;
  w[1] = nb;
  w[2] = mtot;
  int moff = 0;
  for (int q = 0; q < nb; ++q) {
    w[3 + 3 * q] = first[q];
    w[4 + 3 * q] = size[q];
    w[5 + 3 * q] = moff;
    moff += size[q] * size[q];
  }
  for (int r = 0; r < nl; ++r) {
    uint8_t mem[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t signs = 0;
    for (size_t q = 0; q < rows[r].mem.size(); ++q) {
      mem[q] = (uint8_t)rows[r].mem[q];
      if (rows[r].sgn[q] < 0) signs |= 1u << q;
    }
    std::memcpy(&w[rows_at() + 3 * r], mem, 8);
    w[rows_at() + 3 * r + 2] = (uint32_t)rows[r].mem.size() | signs << 8 | (uint32_t)blk[r] << 16;
  }
  for (int e = 0; e < nl; ++e) {
    uint8_t rr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t signs = 0, cnt = 0;
    for (int r = 0; r < nl; ++r)
      for (size_t q = 0; q < rows[r].mem.size(); ++q)
        if (rows[r].mem[q] == e) {
          rr[cnt] = (uint8_t)r;
          if (rows[r].sgn[q] < 0) signs |= 1u << cnt;
          ++cnt;
        }
    if (cnt == 0 || cnt > 8) return false;
    std::memcpy(&w[edges_at(nl) + 3 * e], rr, 8);
    w[edges_at(nl) + 3 * e + 2] = cnt | signs << 8;
  }
  float* mh = reinterpret_cast<float*>(w + m_at(nl));
  float* ml = mh + mtot;
  for (int q = 0; q < nb; ++q)
    for (int r = 0; r < size[q]; ++r)
      for (int s = 0; s < size[q]; ++s) {
        const int R = first[q] + r, S = first[q] + s;
        const double v = Bt[(size_t)R * nl + S] / ((double)rows[R].mem.size() * rows[S].mem.size());
        const float hi = (float)v;
        const int o = (int)w[5 + 3 * q] + s * size[q] + r;  // column-major: a warp reads consecutive rows
        mh[o] = hi;
        ml[o] = (float)(v - (double)hi);
      }
  return true;
}

namespace {

// global index of edge (d, i, j, k) (layout of ndmg.h) and its affine part
__device__ __forceinline__ int64_t sym_edge_gidx(int n, int d, int i, int j, int k) {
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  if (d == 0) return ((int64_t)(k - 1) * (n - 1) + (j - 1)) * n + i;
  if (d == 1) return N3 + ((int64_t)(k - 1) * n + j) * (n - 1) + (i - 1);
  return 2 * N3 + ((int64_t)k * (n - 1) + (j - 1)) * (n - 1) + (i - 1);
}
__device__ __forceinline__ int sym_edge_lin(int n, int d, int i, int j, int k) {
  return d == 0 ? i + n * j + n * (n - 1) * k : d == 1 ? i + (n - 1) * j + n * (n - 1) * k
                                                     : i + (n - 1) * j + (n - 1) * (n - 1) * k;
}

constexpr int kSymThreads = 256;
constexpr int kSymPB = 16;  // patches per pass, 8 per thread half
// row strides of the per-pass arrays: an odd number of 16-byte slots, so the
// 16-byte accesses of 8 consecutive rows (one shared-memory wavefront) fall
// into distinct slots
constexpr int kRS64 = kSymPB + 2;  // int64 entries per row of I64
constexpr int kRS32 = kSymPB + 4;  // floats per row of Th, Tl, Oh, Ol

__host__ __device__ constexpr size_t sym_region_a(int nl) {  // I64, then Oh / Ol over it
  return (size_t)nl * kRS64 * 8 > (size_t)nl * kRS32 * 8 ? (size_t)nl * kRS64 * 8 : (size_t)nl * kRS32 * 8;
}

// v 2^s truncated to int64 on the integer pipe (|v| 2^s < 2^62)
__device__ __forceinline__ long long scaled_fixed(double v, int s) {
  const long long bits = __double_as_longlong(v);
  const int e = (int)((bits >> 52) & 0x7FF);
  const long long m = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
  const int sh = e - 1075 + s;
  long long r = sh >= 0 ? (m << sh) : (sh > -63 ? (m >> -sh) : 0LL);
  r = e == 0 ? 0LL : r;
  return bits < 0 ? -r : r;
}

// an int64 as a pair of floats hi + lo holding its top 48 bits
__device__ __forceinline__ void fixed_pair(long long t, float& hi, float& lo) {
  const unsigned sign = t < 0 ? 0x80000000u : 0u;
  unsigned long long a = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
  if (a == 0ull) {
    hi = lo = 0.f;
    return;
  }
  const int lz = __clzll((long long)a);
  const int E = 63 - lz;  // exponent of the leading one
  a <<= lz;
  hi = __uint_as_float(sign | ((unsigned)(E + 127) << 23) | ((unsigned)(a >> 40) & 0x7FFFFFu));
  const float l24 = __uint2float_rn((unsigned)(a >> 16) & 0xFFFFFFu);  // exact (< 2^24)
  lo = (sign ? -l24 : l24) * __uint_as_float((unsigned)(E - 47 + 127) << 23);
}

__device__ __forceinline__ double pair_to_double(float h, float l) {
  auto f2d = [](float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned ef = (u >> 23) & 0xFFu;
    const unsigned long long bits =
        ef == 0u ? s
                 : (ef == 0xFFu ? 0x7FF8000000000000ull
                                : s | ((unsigned long long)(ef + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29));
    return __longlong_as_double((long long)bits);
  };
  return f2d(h) + f2d(l);
}

// (sh, sl) += d * (rh + rl) with d = dh + dl: exact product error by fma,
// error-free two-sum into sh, errors and cross terms into sl
__device__ __forceinline__ void df_fma(float dh, float dl, float rh, float rl, float& sh, float& sl) {
  const float prod = __fmul_rn(dh, rh);
  const float err = fmaf(dh, rh, -prod);
  const float low = fmaf(dh, rl, fmaf(dl, rh, err));
  const float t = __fadd_rn(sh, prod);
  const float bb = __fsub_rn(t, sh);
  const float e2 = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(prod, bb));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(e2, low));
}

// (sh, sl) += (xh + xl)
__device__ __forceinline__ void df_add(float xh, float xl, float& sh, float& sl) {
  const float t = __fadd_rn(sh, xh);
  const float bb = __fsub_rn(t, sh);
  const float e2 = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(xh, bb));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(e2, xl));
}

// CTAs [gp, gridDim.x) (gp < gridDim.x only when Ainv is given) take the
// 6 x 6 interior-space solves of the coarse elements instead, kSymThreads
// elements per CTA, with atomic additions (vertex patches contain
// element-interior edges)
__device__ __forceinline__ void interior_solves64(int n, int blk, const double* __restrict__ Ainv, double eta,
                                                  const double* __restrict__ r, double* __restrict__ z) {
  __shared__ double As[36];
  if (threadIdx.x < 36) As[threadIdx.x] = __ldg(Ainv + threadIdx.x);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();
  const int nc = n / 2;
  const int64_t NT = (int64_t)nc * nc * nc;
  const int64_t t = (int64_t)blk * blockDim.x + threadIdx.x;
  if (t >= NT) return;
  const int I = (int)(t % nc), J = (int)((t / nc) % nc), K = (int)(t / ((int64_t)nc * nc));
  int64_t g[6];
  int q = 0;
  for (int d = 0; d < 3; ++d)
    for (int s2 = 0; s2 < 2; ++s2) {
      int pq[3] = {2 * I + 1, 2 * J + 1, 2 * K + 1};
      pq[d] = (d == 0 ? 2 * I : d == 1 ? 2 * J : 2 * K) + s2;
      g[q++] = sym_edge_gidx(n, d, pq[0], pq[1], pq[2]);
    }
  double rv[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) rv[a] = __ldg(r + g[a]);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    double sum = 0.0;
#pragma unroll
    for (int b = 0; b < 6; ++b) sum = fma(As[a * 6 + b], rv[b], sum);
    atomicAdd(z + g[a], eta * sum);
  }
}

__global__ void __launch_bounds__(kSymThreads, 3) k_patch_sym(int n, PatchFamily fam, const uint32_t* __restrict__ blob,
                                                              int blob_words, double eta, const double* __restrict__ r,
                                                              double* __restrict__ z, const double* __restrict__ Ainv,
                                                              int gp) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if ((int)blockIdx.x >= gp) {
    const int64_t N3b = (int64_t)n * (n - 1) * (n - 1);
    interior_solves64(n, (int)blockIdx.x - gp, Ainv, eta, r + (int64_t)blockIdx.y * 3 * N3b,
                      z + (int64_t)blockIdx.y * 3 * N3b);
    return;
  }
  constexpr int H = kSymPB / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nl = fam.nloc;
  uint32_t* W = reinterpret_cast<uint32_t*>(smem_raw);                        // the blob
  unsigned char* regA = smem_raw + ((blob_words * 4 + 15) / 16) * 16;
  long long* I64 = reinterpret_cast<long long*>(regA);  // nl rows of kRS64
  float* Oh = reinterpret_cast<float*>(regA);            // over I64 once T is applied: nl rows of kRS32
  float* Ol = Oh + nl * kRS32;
  float* Th = reinterpret_cast<float*>(regA + sym_region_a(nl));  // nl rows of kRS32
  float* Tl = Th + nl * kRS32;
  unsigned* loff = reinterpret_cast<unsigned*>(Tl + nl * kRS32);
  long long* pbase = reinterpret_cast<long long*>(loff + ((nl + 1) & ~1));
  unsigned* amax = reinterpret_cast<unsigned*>(pbase + 3 * kSymPB);
  const int tid = threadIdx.x;
  // set-up, independent of the previous kernel: the blob and the local offsets
  for (int q = tid; q < blob_words; q += blockDim.x) W[q] = __ldg(blob + q);
  const int bx = fam.b[0], by = fam.b[1], bz = fam.b[2];
  const int cx = bx * (by - 1) * (bz - 1), cy = (bx - 1) * by * (bz - 1);
  for (int l = tid; l < nl; l += blockDim.x) {
    int d, i, j, k, e = l;
    if (e < cx) {
      d = 0; i = e % bx; j = (e / bx) % (by - 1) + 1; k = e / (bx * (by - 1)) + 1;
    } else if ((e -= cx) < cy) {
      d = 1; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % by; k = e / ((bx - 1) * by) + 1;
    } else {
      e -= cy;
      d = 2; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % (by - 1) + 1; k = e / ((bx - 1) * (by - 1));
    }
    loff[l] = (unsigned)sym_edge_lin(n, d, i, j, k) | ((unsigned)d << 30);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  r += (int64_t)blockIdx.y * 3 * N3;
  z += (int64_t)blockIdx.y * 3 * N3;
  __syncthreads();
  const int half = tid / 128, row = tid % 128;
  const bool active = row < nl;
  const int my_off = active ? (int)(loff[row] & 0x3FFFFFFFu) : 0, my_d = active ? (int)(loff[row] >> 30) : 0;
  // this thread's row of T, its block of M, and its edge's rows of T^t
  uint32_t rw0 = 0, rw1 = 0, rw2 = 0, ew0 = 0, ew1 = 0, ew2 = 0;
  int b0 = 0, bs = 0, mo = 0;
  if (active) {
    rw0 = W[rows_at() + 3 * row];
    rw1 = W[rows_at() + 3 * row + 1];
    rw2 = W[rows_at() + 3 * row + 2];
    ew0 = W[edges_at(nl) + 3 * row];
    ew1 = W[edges_at(nl) + 3 * row + 1];
    ew2 = W[edges_at(nl) + 3 * row + 2];
    const int q = (int)(rw2 >> 16);
    b0 = (int)W[3 + 3 * q];
    bs = (int)W[4 + 3 * q];
    mo = (int)W[5 + 3 * q] + (row - b0);
  }
  const float* Mh = reinterpret_cast<const float*>(W + m_at(nl));
  const float* Ml = Mh + W[2];
  const int64_t NP = (int64_t)fam.np[0] * fam.np[1] * fam.np[2];
  for (int64_t base = (int64_t)blockIdx.x * kSymPB; base < NP; base += (int64_t)gp * kSymPB) {
    if (tid < kSymPB * 3) {
      const int pp = tid / 3, d = tid % 3;
      const int64_t P = base + pp < NP ? base + pp : NP - 1;
      const int pa = (int)(P % fam.np[0]) + fam.p0[0];
      const int pb = (int)((P / fam.np[0]) % fam.np[1]) + fam.p0[1];
      const int pc = (int)(P / ((int64_t)fam.np[0] * fam.np[1])) + fam.p0[2];
      pbase[tid] = sym_edge_gidx(n, d, fam.stride * pa - fam.shift[0], fam.stride * pb - fam.shift[1],
                                 fam.stride * pc - fam.shift[2]);
    }
    if (tid == 0) *amax = 0u;
    __syncthreads();
    // gather (thread (half, row): local edge `row` of the half's 8 patches)
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
    if ((tid & 31) == 0) atomicMax(amax, m);
    __syncthreads();
    // fixed point: the pass maximum lies in [2^52, 2^53); Inf or NaN make
    // the whole pass NaN
    const unsigned mw = *amax;
    const bool bad = mw >= 0x7FF00000u;
    const int ex = mw == 0 ? 0 : (int)(mw >> 20) - 1023;
    if (active) {
#pragma unroll
      for (int p = 0; p < H; p += 2) {
        longlong2 v2;
        v2.x = scaled_fixed(rv[p], 52 - ex);
        v2.y = scaled_fixed(rv[p + 1], 52 - ex);
        *reinterpret_cast<longlong2*>(I64 + row * kRS64 + half * H + p) = v2;
      }
    }
    __syncthreads();
    // t = T r (exact), as float pairs
    if (active) {
      const int cnt = (int)(rw2 & 0xFFu);
      const uint32_t sg = (rw2 >> 8) & 0xFFu;
      long long t[H];
#pragma unroll
      for (int p = 0; p < H; ++p) t[p] = 0;
      for (int q = 0; q < cnt; ++q) {
        const int mem = (int)(((q < 4 ? rw0 : rw1) >> (8 * (q & 3))) & 0xFFu);
        const longlong2* src = reinterpret_cast<const longlong2*>(I64 + mem * kRS64 + half * H);
        const bool neg = (sg >> q) & 1u;
#pragma unroll
        for (int p = 0; p < H / 2; ++p) {
          const longlong2 v2 = src[p];
          t[2 * p] += neg ? -v2.x : v2.x;
          t[2 * p + 1] += neg ? -v2.y : v2.y;
        }
      }
      float th[H], tl[H];
#pragma unroll
      for (int p = 0; p < H; ++p) fixed_pair(t[p], th[p], tl[p]);
      float4* dh = reinterpret_cast<float4*>(Th + row * kRS32 + half * H);
      float4* dl = reinterpret_cast<float4*>(Tl + row * kRS32 + half * H);
      dh[0] = make_float4(th[0], th[1], th[2], th[3]);
      dh[1] = make_float4(th[4], th[5], th[6], th[7]);
      dl[0] = make_float4(tl[0], tl[1], tl[2], tl[3]);
      dl[1] = make_float4(tl[4], tl[5], tl[6], tl[7]);
    }
    __syncthreads();
    // o = M t on this row's block (double-float), over I64
    if (active) {
      float sh[H], sl[H];
#pragma unroll
      for (int p = 0; p < H; ++p) sh[p] = sl[p] = 0.f;
      for (int c = 0; c < bs; ++c) {
        const float dh = Mh[mo + c * bs], dl = Ml[mo + c * bs];
        const float4* th4 = reinterpret_cast<const float4*>(Th + (b0 + c) * kRS32 + half * H);
        const float4* tl4 = reinterpret_cast<const float4*>(Tl + (b0 + c) * kRS32 + half * H);
        const float4 h0 = th4[0], h1 = th4[1], l0 = tl4[0], l1 = tl4[1];
        const float rh[H] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
        const float rl[H] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
#pragma unroll
        for (int p = 0; p < H; ++p) df_fma(dh, dl, rh[p], rl[p], sh[p], sl[p]);
      }
      float4* oh = reinterpret_cast<float4*>(Oh + row * kRS32 + half * H);
      float4* ol = reinterpret_cast<float4*>(Ol + row * kRS32 + half * H);
      oh[0] = make_float4(sh[0], sh[1], sh[2], sh[3]);
      oh[1] = make_float4(sh[4], sh[5], sh[6], sh[7]);
      ol[0] = make_float4(sl[0], sl[1], sl[2], sl[3]);
      ol[1] = make_float4(sl[4], sl[5], sl[6], sl[7]);
    }
    __syncthreads();
    // y = T^t o for this thread's edge, back to FP64 and into z
    if (active) {
      const int cnt = (int)(ew2 & 0xFFu);
      const uint32_t sg = (ew2 >> 8) & 0xFFu;
      float yh[H], yl[H];
#pragma unroll
      for (int p = 0; p < H; ++p) yh[p] = yl[p] = 0.f;
      for (int q = 0; q < cnt; ++q) {
        const int rr = (int)(((q < 4 ? ew0 : ew1) >> (8 * (q & 3))) & 0xFFu);
        const float sgn = ((sg >> q) & 1u) ? -1.f : 1.f;
        const float4* oh = reinterpret_cast<const float4*>(Oh + rr * kRS32 + half * H);
        const float4* ol = reinterpret_cast<const float4*>(Ol + rr * kRS32 + half * H);
        const float4 h0 = oh[0], h1 = oh[1], l0 = ol[0], l1 = ol[1];
        const float xh[H] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
        const float xl[H] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
#pragma unroll
        for (int p = 0; p < H; ++p) df_add(sgn * xh[p], sgn * xl[p], yh[p], yl[p]);
      }
      const double back = ldexp(eta, ex - 52);
#pragma unroll
      for (int p = 0; p < H; ++p) {
        const int pp = half * H + p;
        if (base + pp < NP)
          atomicAdd(z + pbase[3 * pp + my_d] + my_off, bad ? (double)NAN : back * pair_to_double(yh[p], yl[p]));
      }
    }
    __syncthreads();  // pbase, I64 / Oh / Ol and Th / Tl are rewritten by the next pass
  }
}

// The FP32 smoother correction of eq. (Preconditioner P) in the same basis,
// with the interior solves in the same launch: CTAs [0, npb) take PB vertex
// patches each (gather, T, the FP32 block products, T^t, atomic additions
// into z), the other CTAs take the 6 x 6 interior solves of 128 coarse
// elements each.  The tables and the float blocks of M are copied into
// shared memory before the kernel waits for its predecessor (they are
// constant); a CTA's critical path is then one gather and a seventh of the
// dense product's multiply-adds.
constexpr int kSym32PB = 8;
constexpr int kRS8 = kSym32PB + 4;  // floats per row: an odd number of 16-byte slots

template <int PB>
__global__ void __launch_bounds__(128) k_smooth_sym32(int n, PatchFamily fam, const uint32_t* __restrict__ blob,
                                                      int blob_words, const float* __restrict__ Ainv, float eta,
                                                      int npb, const float* __restrict__ r, float* __restrict__ z) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  static_assert(PB == 8, "the 16-byte accesses below take 8 patches per row");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned loff[128];
  __shared__ long long pbase[3 * PB];
  __shared__ float As[36];
  const int tid = threadIdx.x;
  const int64_t N3 = (int64_t)n * (n - 1) * (n - 1);
  if ((int)blockIdx.x < npb) {
    const int nl = fam.nloc;
    uint32_t* W = reinterpret_cast<uint32_t*>(smem_raw);
    const int wpad = (blob_words + 3) & ~3;  // the blob is stored padded to 16 bytes
    float* Rr = reinterpret_cast<float*>(W + wpad);  // nl rows of kRS8
    float* Tt = Rr + nl * kRS8;
    float* Oo = Tt + nl * kRS8;
    {
      const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(W));
      const uint4* src = reinterpret_cast<const uint4*>(blob);
      for (int q = tid; q < wpad / 4; q += blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16u * q), "l"(src + q) : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const int bx = fam.b[0], by = fam.b[1], bz = fam.b[2];
    const int cx = bx * (by - 1) * (bz - 1), cy = (bx - 1) * by * (bz - 1);
    if (tid < nl) {
      int d, i, j, k, e = tid;
      if (e < cx) {
        d = 0; i = e % bx; j = (e / bx) % (by - 1) + 1; k = e / (bx * (by - 1)) + 1;
      } else if ((e -= cx) < cy) {
        d = 1; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % by; k = e / ((bx - 1) * by) + 1;
      } else {
        e -= cy;
        d = 2; i = e % (bx - 1) + 1; j = (e / (bx - 1)) % (by - 1) + 1; k = e / ((bx - 1) * (by - 1));
      }
      loff[tid] = (unsigned)sym_edge_lin(n, d, i, j, k) | ((unsigned)d << 30);
    }
    const int64_t NP = (int64_t)fam.np[0] * fam.np[1] * fam.np[2];
    const int64_t base = (int64_t)blockIdx.x * PB;
    if (tid < 3 * PB) {
      const int pp = tid / 3, d = tid % 3;
      const int64_t P = base + pp < NP ? base + pp : NP - 1;
      const int pa = (int)(P % fam.np[0]) + fam.p0[0];
      const int pb = (int)((P / fam.np[0]) % fam.np[1]) + fam.p0[1];
      const int pc = (int)(P / ((int64_t)fam.np[0] * fam.np[1])) + fam.p0[2];
      pbase[tid] = sym_edge_gidx(n, d, fam.stride * pa - fam.shift[0], fam.stride * pb - fam.shift[1],
                                 fam.stride * pc - fam.shift[2]);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    r += (int64_t)blockIdx.y * 3 * N3;
    z += (int64_t)blockIdx.y * 3 * N3;
    __syncthreads();
    const bool active = tid < nl;
    const int row = tid;
    const int my_off = active ? (int)(loff[row] & 0x3FFFFFFFu) : 0, my_d = active ? (int)(loff[row] >> 30) : 0;
    if (active) {
      float v[PB];
#pragma unroll
      for (int p = 0; p < PB; ++p) v[p] = base + p < NP ? __ldg(r + pbase[3 * p + my_d] + my_off) : 0.f;
      float4* d4 = reinterpret_cast<float4*>(Rr + row * kRS8);
      d4[0] = make_float4(v[0], v[1], v[2], v[3]);
      d4[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    uint32_t rw0 = 0, rw1 = 0, rw2 = 0;
    int b0 = 0, bs = 0, mo = 0;
    if (active) {
      rw0 = W[rows_at() + 3 * row];
      rw1 = W[rows_at() + 3 * row + 1];
      rw2 = W[rows_at() + 3 * row + 2];
      const int q = (int)(rw2 >> 16);
      b0 = (int)W[3 + 3 * q];
      bs = (int)W[4 + 3 * q];
      mo = (int)W[5 + 3 * q] + (row - b0);
      // t = T r
      const int cnt = (int)(rw2 & 0xFFu);
      const uint32_t sg = (rw2 >> 8) & 0xFFu;
      float t[PB];
#pragma unroll
      for (int p = 0; p < PB; ++p) t[p] = 0.f;
      for (int q2 = 0; q2 < cnt; ++q2) {
        const int mem = (int)(((q2 < 4 ? rw0 : rw1) >> (8 * (q2 & 3))) & 0xFFu);
        const float sgn = ((sg >> q2) & 1u) ? -1.f : 1.f;
        const float4* s4 = reinterpret_cast<const float4*>(Rr + mem * kRS8);
        const float4 a0 = s4[0], a1 = s4[1];
        t[0] = fmaf(sgn, a0.x, t[0]); t[1] = fmaf(sgn, a0.y, t[1]); t[2] = fmaf(sgn, a0.z, t[2]); t[3] = fmaf(sgn, a0.w, t[3]);
        t[4] = fmaf(sgn, a1.x, t[4]); t[5] = fmaf(sgn, a1.y, t[5]); t[6] = fmaf(sgn, a1.z, t[6]); t[7] = fmaf(sgn, a1.w, t[7]);
      }
      float4* d4 = reinterpret_cast<float4*>(Tt + row * kRS8);
      d4[0] = make_float4(t[0], t[1], t[2], t[3]);
      d4[1] = make_float4(t[4], t[5], t[6], t[7]);
    }
    __syncthreads();
    if (active) {
      // o = M t on this row's block
      const float* Mh = reinterpret_cast<const float*>(W + m_at(nl));
      float o[PB];
#pragma unroll
      for (int p = 0; p < PB; ++p) o[p] = 0.f;
      for (int c = 0; c < bs; ++c) {
        const float m = Mh[mo + c * bs];
        const float4* s4 = reinterpret_cast<const float4*>(Tt + (b0 + c) * kRS8);
        const float4 a0 = s4[0], a1 = s4[1];
        o[0] = fmaf(m, a0.x, o[0]); o[1] = fmaf(m, a0.y, o[1]); o[2] = fmaf(m, a0.z, o[2]); o[3] = fmaf(m, a0.w, o[3]);
        o[4] = fmaf(m, a1.x, o[4]); o[5] = fmaf(m, a1.y, o[5]); o[6] = fmaf(m, a1.z, o[6]); o[7] = fmaf(m, a1.w, o[7]);
      }
      float4* d4 = reinterpret_cast<float4*>(Oo + row * kRS8);
      d4[0] = make_float4(o[0], o[1], o[2], o[3]);
      d4[1] = make_float4(o[4], o[5], o[6], o[7]);
    }
    __syncthreads();
    if (active) {
      // y = T^t o for this thread's edge, into z
      const uint32_t ew0 = W[edges_at(nl) + 3 * row], ew1 = W[edges_at(nl) + 3 * row + 1];
      const uint32_t ew2 = W[edges_at(nl) + 3 * row + 2];
      const int cnt = (int)(ew2 & 0xFFu);
      const uint32_t sg = (ew2 >> 8) & 0xFFu;
      float y[PB];
#pragma unroll
      for (int p = 0; p < PB; ++p) y[p] = 0.f;
      for (int q2 = 0; q2 < cnt; ++q2) {
        const int rr = (int)(((q2 < 4 ? ew0 : ew1) >> (8 * (q2 & 3))) & 0xFFu);
        const float sgn = ((sg >> q2) & 1u) ? -1.f : 1.f;
        const float4* s4 = reinterpret_cast<const float4*>(Oo + rr * kRS8);
        const float4 a0 = s4[0], a1 = s4[1];
        y[0] = fmaf(sgn, a0.x, y[0]); y[1] = fmaf(sgn, a0.y, y[1]); y[2] = fmaf(sgn, a0.z, y[2]); y[3] = fmaf(sgn, a0.w, y[3]);
        y[4] = fmaf(sgn, a1.x, y[4]); y[5] = fmaf(sgn, a1.y, y[5]); y[6] = fmaf(sgn, a1.z, y[6]); y[7] = fmaf(sgn, a1.w, y[7]);
      }
#pragma unroll
      for (int p = 0; p < PB; ++p)
        if (base + p < NP) atomicAdd(z + pbase[3 * p + my_d] + my_off, eta * y[p]);
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
      int pq[3] = {2 * I + 1, 2 * J + 1, 2 * K + 1};
      pq[d] = (d == 0 ? 2 * I : d == 1 ? 2 * J : 2 * K) + s2;
      g[q++] = sym_edge_gidx(n, d, pq[0], pq[1], pq[2]);
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

}  // namespace

size_t smooth_sym32_smem(int nloc, int blob_words) {
  return sizeof(uint32_t) * ((blob_words + 3) & ~3) + sizeof(float) * 3 * nloc * kRS8;
}

cudaError_t prepare_smooth_sym32() {
  return cudaFuncSetAttribute(k_smooth_sym32<kSym32PB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
}

void launch_smooth_sym32(cudaStream_t s, int n, const uint32_t* blob, int blob_words, const float* Ainv, double eta,
                         const float* r, float* z, int R) {
  const PatchFamily fam = vertex_family(n);
  const int64_t NP = (int64_t)fam.np[0] * fam.np[1] * fam.np[2];
  if (NP <= 0) return;
  const int64_t nc = n / 2;
  const int npb = (int)((NP + kSym32PB - 1) / kSym32PB);
  const int nbb = (int)((nc * nc * nc + 127) / 128);
  launch_pdl(k_smooth_sym32<kSym32PB>, dim3(npb + nbb, R), 128, smooth_sym32_smem(fam.nloc, blob_words), s, n, fam,
             blob, blob_words, Ainv, (float)eta, npb, r, z);
}

size_t patch_sym_smem(int nloc, int blob_words) {
  return (size_t)((blob_words * 4 + 15) / 16) * 16 + sym_region_a(nloc) + sizeof(float) * 2 * nloc * kRS32 +
         sizeof(int) * ((nloc + 1) & ~1) + sizeof(long long) * 3 * kSymPB + 16;
}

cudaError_t prepare_patch_sym() {
  return cudaFuncSetAttribute(k_patch_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
}

void launch_patch_sym(cudaStream_t s, int sm, int n, const PatchFamily& fam, const uint32_t* blob, int blob_words,
                      double eta, const double* r, double* z, int R, const double* Ainv) {
  const int64_t NP = (int64_t)fam.np[0] * fam.np[1] * fam.np[2];
  if (NP <= 0 && !Ainv) return;
  int64_t blocks = (NP + kSymPB - 1) / kSymPB;
  const int64_t cap = (int64_t)sm * 3;
  if (blocks > cap) blocks = cap;
  const int64_t nc = n / 2;
  const int64_t nbb = Ainv ? (nc * nc * nc + kSymThreads - 1) / kSymThreads : 0;
  launch_pdl(k_patch_sym, dim3((int)(blocks + nbb), R), kSymThreads, patch_sym_smem(fam.nloc, blob_words), s, n, fam,
             blob, blob_words, eta, r, z, Ainv, (int)blocks);
}

}  // namespace ndmg
