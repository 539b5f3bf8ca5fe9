// Smoother correction of eq. (Preconditioner P) on the 5th-gen tensor cores
// in a cell-owned form (sm_103a, tcgen05 + TMEM):
//
//     z += eta * ( sum_T J_T A_T^{-1} J_T^t r  +  sum_V J_V W W^t J_V^t r ),
//
// W the 108 x 60 Gram factor of the vertex-space operator, the same for
// every interior coarse vertex V (constant alpha, uniform grid).
//
// Every fine edge is owned by one coarse cell: the cell C = (i, j, k) >> 1 of
// its lowest fine node (i, j, k), at one of 24 slots (direction d, node
// parities a, b, c).  The 108 edges of the vertex patch of V are owned by the
// 8 cells V + o, o in {-1, 0}^3, so with R_C the 24 owned values of r at cell
// C and W'_o the rows of W that cell V + o holds (zero where a slot is not in
// the patch),
//
//     t_V   = sum_{o in {-1,0}^3} W'_o^t R_{V+o}                (60 values)
//     out_C = sum_{o in {0,1}^3}  W'_{-o} t_{C+o}               (24 values)
//
// i.e. the patch gather and the overlapping scatter become sums over
// neighbouring rows.  With R and t stored row by row (cells / vertices of a
// 16 x 16 layer tile, x fastest, rows 16 bytes apart within a K-slice), the
// neighbour C + o is the same matrix at a row offset o_x + 16 o_y and the
// layer of o_z, so each term is one tcgen05.mma whose A descriptor simply
// starts o_x + 16 o_y rows further; no operand is gathered or scattered.
//
// A CTA (persistent, one per SM) takes work items = a column of 16 x 16
// cells (the inner 14 x 14 owned, one halo cell each side) over a chunk of
// cell layers along z and streams up the layers:
//   1. r of the next cell layer is loaded straight into registers (a layer
//      ahead), scaled by a power of two so that max |r| <= 1 on the layer
//      tile, rounded to fp16 / bf16 and stored as rows of R (3 K-slices of 8
//      slots); the interior-space values stay in FP32 registers;
//   2. GEMM1: t of vertex layer kv from R of cell layers kv-1 and kv (two
//      FP32 accumulators in TMEM, one per layer, so each layer keeps its own
//      scale), 12 MMAs per M = 128 tile (only the K-slices a neighbour can
//      hold);
//   3. t is combined in FP32, zeroed on boundary vertices, rescaled, rounded
//      and stored as rows (8 K-slices);
//   4. GEMM2: out of cell layer kv-1 from t of vertex layers kv-1, kv (N = 32
//      or 16 per neighbour);
//   5. each thread owns one cell row: it reads out from TMEM, adds the 6 x 6
//      interior-space solve in FP32 and adds eta * out to the cell's owned
//      edges of z (every edge is written by exactly one thread of one CTA:
//      no atomics).
// Steps of consecutive layers overlap: GEMM1 of a layer runs while the
// previous layer's output is written out, GEMM2 while the next layer is
// staged.
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "tc_cell.cuh"
#include "tc_common.cuh"
#include "pdl.cuh"

namespace ndmg {
namespace {
using namespace tc;

constexpr int kTile = 16;                    // cells (and vertices) per axis of a layer tile
constexpr int kOwn = kTile - 2;              // owned cells per axis
constexpr int kRows = kTile * kTile;         // 256 rows: two M = 128 tiles
constexpr int kThreads = 512;                // thread t: row t & 255, half t >> 8
constexpr int kShift = kTile + 1;            // largest row offset of a neighbour
constexpr int kRowsR = kRows + kShift;       // R rows -kShift .. kRows - 1
constexpr int kRowsT = kRows + kShift;       // t rows 0 .. kRows + kShift - 1
constexpr uint32_t LBO_R = kRowsR * 16;      // bytes between K-slices of one R layer
constexpr uint32_t LBO_T = kRowsT * 16;
constexpr uint32_t R_LAYER = 3 * LBO_R;      // 24 slots = 3 K-slices
constexpr uint32_t T_LAYER = 8 * LBO_T;      // 64 t components = 8 K-slices
constexpr uint32_t kTmemCols = 512;          // per M-tile q: T_lo, T_hi (64 each), O_0, O_1 (32 each) at 192 q

// The 24 slots of a cell, grouped into three K-slices so that every
// neighbour offset needs at most two MMAs of K = 16: slot = d | a << 2 |
// b << 3 | c << 4 (direction, parities of the lowest node).  S0 holds the 6
// interior-space edges (positions 0..5, in the order of the 6 x 6 interior
// operator: x segment 0, 1, y 0, 1, z 0, 1) and the z-edges with x, y parity
// 0; S1 and S2 the rest.  Packed 5 bits per position, 12 positions a word.
__host__ __device__ constexpr uint64_t pslot(int d, int a, int b, int c) {
  return (uint64_t)(d | a << 2 | b << 3 | c << 4);
}
constexpr uint64_t kPosLo =
    pslot(0, 0, 1, 1) | pslot(0, 1, 1, 1) << 5 | pslot(1, 1, 0, 1) << 10 | pslot(1, 1, 1, 1) << 15 |
    pslot(2, 1, 1, 0) << 20 | pslot(2, 1, 1, 1) << 25 | pslot(2, 0, 0, 0) << 30 | pslot(2, 0, 0, 1) << 35 |
    pslot(0, 0, 1, 0) << 40 | pslot(0, 1, 1, 0) << 45 | pslot(1, 1, 0, 0) << 50 | pslot(1, 1, 1, 0) << 55;
constexpr uint64_t kPosHi =
    pslot(1, 0, 0, 1) | pslot(1, 0, 1, 1) << 5 | pslot(2, 0, 1, 0) << 10 | pslot(2, 0, 1, 1) << 15 |
    pslot(0, 0, 0, 1) << 20 | pslot(0, 1, 0, 1) << 25 | pslot(2, 1, 0, 0) << 30 | pslot(2, 1, 0, 1) << 35 |
    pslot(0, 0, 0, 0) << 40 | pslot(0, 1, 0, 0) << 45 | pslot(1, 0, 0, 0) << 50 | pslot(1, 0, 1, 0) << 55;
__host__ __device__ constexpr int pos_slot(int p) {
  return (int)((p < 12 ? kPosLo >> (5 * p) : kPosHi >> (5 * (p - 12))) & 31u);
}
__host__ __device__ constexpr int slot_d(int s) { return s & 3; }
__host__ __device__ constexpr int slot_par(int s, int axis) { return (s >> (2 + axis)) & 1; }
// axes across the slot's direction whose node parity is 0: a neighbour with
// offset -1 (GEMM1) / +1 (GEMM2) along such an axis does not hold the edge
__host__ __device__ constexpr int slot_zero_mask(int s) {
  int m = 0;
  for (int e = 0; e < 3; ++e)
    if (e != slot_d(s) && slot_par(s, e) == 0) m |= 1 << e;
  return m;
}

// GEMM1 plan per neighbour J (bit e set: offset -1 along axis e): the
// K-slice pairs of its MMAs.  Two MMAs (S0,S1), (S1,S2) when the neighbour
// holds slots of all three slices (the second MMA's S1 rows are zero), one
// otherwise.
__host__ __device__ constexpr int g1_count(int J) { return (J == 0 || J == 1 || J == 2 || J == 4) ? 2 : 1; }
__host__ __device__ constexpr int g1_first(int J, int i) { return i == 0 ? 0 : 1; }
__host__ __device__ constexpr int g1_second(int J, int i) { return i == 1 ? 2 : (J == 5 ? 2 : 1); }
__host__ __device__ constexpr int g1_block(int J) {  // first 2 KB block of neighbour J in the GEMM1 image
  int b = 0;
  for (int q = 0; q < J; ++q) b += g1_count(q);
  return b;
}
constexpr int kG1Blocks = g1_block(8);               // 12 blocks of 64 x 16
constexpr int kG1Bytes = kG1Blocks * 64 * 16 * 2;
// GEMM2 per neighbour J (bit e: offset +1 along axis e): N = 16 when its
// outputs all lie in S0, S1 (the first 16 positions), else 32
__host__ __device__ constexpr int g2_n(int J) { return (J == 3 || J == 6 || J == 7) ? 16 : 32; }
__host__ __device__ constexpr int g2_off(int J) {
  int b = 0;
  for (int q = 0; q < J; ++q) b += g2_n(q) * 64 * 2;
  return b;
}
constexpr int kG2Bytes = g2_off(8);
constexpr int kImgBytes = kG1Bytes + kG2Bytes;       // both images, then the float 1 / s_w^2
constexpr int kImgTotal = kImgBytes + 16;

// shared memory
constexpr uint32_t OFF_B1 = 0;
constexpr uint32_t OFF_B2 = kG1Bytes;
constexpr uint32_t OFF_R = kImgBytes;                                // 3 layers of R
constexpr uint32_t OFF_T = (OFF_R + 3 * R_LAYER + 127) / 128 * 128;  // 2 layers of t
constexpr uint32_t OFF_BUB = OFF_T + 2 * T_LAYER;                    // FP32 interior-space r: 3 layers x rows x 6
constexpr uint32_t OFF_AT = OFF_BUB + 3 * kRows * 6 * 4;             // 6 x 6 interior inverse (FP32)
constexpr uint32_t OFF_SC = OFF_AT + 36 * 4;                         // s[4] (R scales), sigma[4] (t scales)
constexpr uint32_t OFF_RED = OFF_SC + 8 * 4;                         // 16 warp maxima
constexpr uint32_t OFF_BAR = (OFF_RED + 16 * 4 + 7) / 8 * 8;         // mbarriers: GEMM1, GEMM2
constexpr uint32_t OFF_TM = OFF_BAR + 16;                            // TMEM base address
constexpr uint32_t kSmem = OFF_TM + 16;
static_assert(kSmem <= 227 * 1024, "one CTA per SM");
static_assert(OFF_R % 16 == 0 && OFF_T % 16 == 0 && OFF_B2 % 16 == 0, "descriptor alignment");
static_assert(LBO_R % 16 == 0 && LBO_T % 16 == 0, "K-slice strides");
static_assert(kImgBytes % 16 == 0, "image copy in 16-byte words");
constexpr int kTimeout = 1;                                          // status code

struct CellArgs {
  int n, nc;
  int ncol, nzc, zlen;       // columns per axis, z chunks, cell layers per chunk
  int items;                 // ncol^2 * nzc * R
  float eta;
  const uint8_t* img;
  const float* AinvT;
  const float* r;
  float* z;
  int* status;
};

// Offset (within one right-hand side, as if on cell layer 0; the layer adds
// kv * stride, 32-bit wrap-around included) of the edge at slot s of cell
// (cx, cy), and whether it is interior as far as x and y decide.  Along z
// the edge is interior on every cell layer of the box except for x- and
// y-edges with node parity 0 on layer 0 (node plane 0).
__host__ __device__ __forceinline__ uint32_t slot_offset(int n, int s, int cx, int cy, bool* ok) {
  const uint32_t n1 = n - 1, N3 = (uint32_t)n * n1 * n1;
  const int d = slot_d(s), a = slot_par(s, 0), b = slot_par(s, 1), c = slot_par(s, 2);
  const int i = 2 * cx + a, j = 2 * cy + b;
  const bool in = cx >= 0 && cy >= 0 && i < n && j < n;
  if (d == 0) {
    *ok = in && j >= 1;
    return ((uint32_t)(c - 1) * n1 + (uint32_t)(j - 1)) * n + (uint32_t)i;
  }
  if (d == 1) {
    *ok = in && i >= 1;
    return N3 + ((uint32_t)(c - 1) * n + (uint32_t)j) * n1 + (uint32_t)(i - 1);
  }
  *ok = in && i >= 1 && j >= 1;
  return 2u * N3 + ((uint32_t)c * n1 + (uint32_t)(j - 1)) * n1 + (uint32_t)(i - 1);
}

// The same offset split into a part that depends only on the slot (and n)
// and the cell's part 2 cx + 2 cy w, w = n for x-edges and n - 1 otherwise
// (kept in registers per thread while the slot part is recomputed on use).
__host__ __device__ __forceinline__ uint32_t slot_const(int n, int s) {
  const uint32_t n1 = n - 1, N3 = (uint32_t)n * n1 * n1;
  const int d = slot_d(s), a = slot_par(s, 0), b = slot_par(s, 1), c = slot_par(s, 2);
  if (d == 0) return ((uint32_t)(c - 1) * n1 + (uint32_t)(b - 1)) * n + (uint32_t)a;
  if (d == 1) return N3 + ((uint32_t)(c - 1) * n + (uint32_t)b) * n1 + (uint32_t)(a - 1);
  return 2u * N3 + ((uint32_t)c * n1 + (uint32_t)(b - 1)) * n1 + (uint32_t)(a - 1);
}

template <bool FP16>
__device__ __forceinline__ void cell_smoother_body(const CellArgs& A) {
  extern __shared__ __align__(128) uint8_t smem[];
  if (*reinterpret_cast<volatile int*>(A.status) != 0) return;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m = tid & (kRows - 1), h = tid >> 8;
  const int u = m & (kTile - 1), v = m >> 4, q = m >> 7;
  const uint32_t lane_base = ((uint32_t)((m & 127) >> 5) * 32u) << 16;  // TMEM lane field of this warp
  const int n = A.n, nc = A.nc;
  const uint32_t n1 = n - 1, N3 = (uint32_t)n * n1 * n1;
  const uint32_t str_xy = 2u * (uint32_t)n * n1, str_z = 2u * n1 * n1;  // per cell layer

  float* At = reinterpret_cast<float*>(smem + OFF_AT);
  float* sc = reinterpret_cast<float*>(smem + OFF_SC);  // sc[kv & 3]: s of R(kv); sc[4 + (kv & 3)]: sigma of t(kv)
  float* red = reinterpret_cast<float*>(smem + OFF_RED);
  const uint32_t bar_g1 = smem_u32(smem + OFF_BAR), bar_g2 = bar_g1 + 8;
  uint32_t* tm_slot = reinterpret_cast<uint32_t*>(smem + OFF_TM);
  const uint32_t sR = smem_u32(smem + OFF_R), sT = smem_u32(smem + OFF_T);
  const uint32_t sB1 = smem_u32(smem + OFF_B1), sB2 = smem_u32(smem + OFF_B2);

  // ---- set-up: TMEM, barriers, operator images (kept for every work item) ----
  if (warp == 0) tmem_alloc(smem_u32(tm_slot), kTmemCols);
  if (tid == 0) {
    mbar_init(bar_g1, 1);
    mbar_init(bar_g2, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    const uint4* src = reinterpret_cast<const uint4*>(A.img);
    uint4* dst = reinterpret_cast<uint4*>(smem + OFF_B1);
    for (int i = tid; i < kImgBytes / 16; i += kThreads) dst[i] = __ldg(src + i);
    // the R and t rings start zeroed (their margin rows feed only rows whose
    // results are never written out, and must hold finite values)
    uint4* ring = reinterpret_cast<uint4*>(smem + OFF_R);
    const int nring = (int)((OFF_T + 2 * T_LAYER - OFF_R) / 16);
    for (int i = tid; i < nring; i += kThreads) ring[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid < 36) At[tid] = __ldg(A.AinvT + tid);
  }
  const float wscale = __ldg(reinterpret_cast<const float*>(A.img + kImgBytes));
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tm_slot;
  const uint32_t tq = tmem + (uint32_t)(192 * q) + lane_base;  // this thread's row of its M-tile
  uint32_t iss1 = 0, iss2 = 0, n1done = 0, n2done = 0;        // MMA groups issued / seen complete
  bool bad = false;
  auto agree = [&]() {
    bad = __syncthreads_or(bad) != 0;
    return bad;
  };

  const uint32_t idesc1 = instr_desc(128, 64, FP16);
  const int NP = h ? 8 : 16;   // positions of this half: 0..15 (S0, S1) or 16..23 (S2)

  for (int item = blockIdx.x; item < A.items && !bad; item += gridDim.x) {
    const int per_rhs = A.ncol * A.ncol * A.nzc;
    const int rhs = item / per_rhs;
    int rem = item - rhs * per_rhs;
    const int zc = rem / (A.ncol * A.ncol);
    rem -= zc * A.ncol * A.ncol;
    const int qy = rem / A.ncol, qx = rem - qy * A.ncol;
    const int k0 = zc * A.zlen, k1 = min(nc, k0 + A.zlen);
    const int cx = kOwn * qx - 1 + u, cy = kOwn * qy - 1 + v;     // this row's cell (and vertex) in x, y
    const bool own_xy = u >= 1 && u <= kOwn && v >= 1 && v <= kOwn && cx < nc && cy < nc;
    const bool vtx_xy = cx >= 1 && cx <= nc - 1 && cy >= 1 && cy <= nc - 1;  // interior coarse vertex
    const float* r = A.r + (size_t)rhs * 3 * N3;
    float* z = A.z + (size_t)rhs * 3 * N3;

    // this thread's positions: bit masks (interior in x, y; x-/y-edge on a
    // node plane of parity 0) and the cell parts of the offsets
    uint32_t okm = 0, c0 = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int s = pos_slot(h ? (16 + (i & 7)) : i);
      bool ok = false;
      slot_offset(n, s, cx, cy, &ok);
      if (i < NP && ok) okm |= 1u << i;
      if (slot_d(s) != 2 && slot_par(s, 2) == 0) c0 |= 1u << i;
    }
    const uint32_t base_x = 2u * (uint32_t)cx + 2u * (uint32_t)cy * (uint32_t)n;
    const uint32_t base_yz = 2u * (uint32_t)cx + 2u * (uint32_t)cy * n1;
    // mask of the positions that are edges of the box on cell layer kv
    auto layer_mask = [&](int kv) -> uint32_t {
      if (kv < 0 || kv >= nc) return 0u;
      return kv == 0 ? (okm & ~c0) : okm;
    };
    auto addr = [&](int i, int kv) -> uint32_t {
      const int s = pos_slot(h ? (16 + (i & 7)) : i);
      const int d = slot_d(s);
      return slot_const(n, s) + (d == 0 ? base_x : base_yz) + (uint32_t)kv * (d == 2 ? str_z : str_xy);
    };

    float cur[16];
    auto load_layer = [&](int kv) {
      const uint32_t lm = layer_mask(kv);
#pragma unroll
      for (int i = 0; i < 16; ++i) cur[i] = ((lm >> i) & 1u) ? __ldg(r + addr(i, kv)) : 0.f;
    };
    load_layer(k0 - 1);
    // interior-space r (FP32) of the last three cell layers, this row's own
    // slots (written and read by the same thread of half 0)
    float* bub = reinterpret_cast<float*>(smem + OFF_BUB) + m * 6;
    auto bub_slot = [&](int layer) { return bub + (((layer % 3) + 3) % 3) * (kRows * 6); };

    // out of cell layer c added into z, in two steps: epi_load issues the
    // loads of this cell's z (before the wait for GEMM2, so that their
    // latency overlaps it), epi_finish reads out from TMEM once GEMM2 is
    // complete and stores z + eta out
    float zv[16];
    auto epi_load = [&](int c) {
      const uint32_t lm = (own_xy && c >= k0 && c < k1) ? layer_mask(c) : 0u;
#pragma unroll
      for (int i = 0; i < 16; ++i) zv[i] = ((lm >> i) & 1u) ? z[addr(i, c)] : 0.f;
    };
    auto epi_finish = [&](int c) {
      const float inv0 = wscale / sc[4 + (c & 3)], inv1 = wscale / sc[4 + ((c + 1) & 3)];
      const uint32_t lm = (own_xy && c >= k0 && c < k1) ? layer_mask(c) : 0u;
#pragma unroll
      for (int grp = 0; grp < 2; ++grp) {
        if (h == 1 && grp == 1) break;
        float o0[8], o1[8];
        const uint32_t col = (uint32_t)(16 * h + 8 * grp);
        tmem_ld8x2(tq + 128 + col, tq + 160 + col, o0, o1);
#pragma unroll
        for (int i = 0; i < 8; ++i) o0[i] = o0[i] * inv0 + o1[i] * inv1;
        if (h == 0 && grp == 0) {
          // interior spaces: positions 0..5 in the order of A_T^{-1}
          const float* rb = bub_slot(c);
          float rbv[6];
#pragma unroll
          for (int x = 0; x < 6; ++x) rbv[x] = rb[x];
#pragma unroll
          for (int w = 0; w < 6; ++w) {
            float s = 0.f;
#pragma unroll
            for (int x = 0; x < 6; ++x) s += At[w * 6 + x] * rbv[x];
            o0[w] += s;
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if ((lm >> (8 * grp + i)) & 1u) z[addr(8 * grp + i, c)] = zv[8 * grp + i] + A.eta * o0[i];
      }
    };

    // R(kv) into ring slot kv mod 3 from the registers (cur = r of layer kv):
    // a block-wide max for the layer's scale, then the rounded rows
    auto stage = [&](int kv) {
      if (h == 0) {
        float* bs = bub_slot(kv);
#pragma unroll
        for (int w = 0; w < 6; ++w) bs[w] = cur[w];
      }
      float amax = 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) amax = fmaxf(amax, fabsf(cur[i]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if ((tid & 31) == 0) red[warp] = amax;
      __syncthreads();
      float mx = 0.f;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) mx = fmaxf(mx, red[w]);
      const float s = mx > 0.f ? exp2f(-ceilf(log2f(mx))) : 1.f;   // power of two: max |s r| <= 1
      if (tid == 0) sc[kv & 3] = s;
      uint8_t* R8 = smem + OFF_R + (uint32_t)((((kv % 3) + 3) % 3) * R_LAYER) + (uint32_t)(m + kShift) * 16u;
      uint4 w0;
      w0.x = pack2<FP16>(cur[0] * s, cur[1] * s);
      w0.y = pack2<FP16>(cur[2] * s, cur[3] * s);
      w0.z = pack2<FP16>(cur[4] * s, cur[5] * s);
      w0.w = pack2<FP16>(cur[6] * s, cur[7] * s);
      *reinterpret_cast<uint4*>(R8 + (uint32_t)(h ? 2 : 0) * LBO_R) = w0;
      if (h == 0) {
        uint4 w1;
        w1.x = pack2<FP16>(cur[8] * s, cur[9] * s);
        w1.y = pack2<FP16>(cur[10] * s, cur[11] * s);
        w1.z = pack2<FP16>(cur[12] * s, cur[13] * s);
        w1.w = pack2<FP16>(cur[14] * s, cur[15] * s);
        *reinterpret_cast<uint4*>(R8 + LBO_R) = w1;
      }
    };
    // GEMM1 (one thread): t of vertex layer kv from R(kv - 1), R(kv)
    auto issue_g1 = [&](int kv) {
      fence_after();
      // descriptors = a base descriptor plus the operand's byte offset / 16
      // in the address field (every address stays below 256 KB)
      const uint32_t slo = sR + (uint32_t)(((kv + 2) % 3) * R_LAYER);   // (kv - 1) mod 3, kv >= 0
      const uint32_t shi = sR + (uint32_t)((((kv % 3) + 3) % 3) * R_LAYER);
      const uint64_t alo = smem_desc(slo, LBO_R, 128), ahi = smem_desc(shi, LBO_R, 128);
      const uint64_t alo2 = smem_desc(slo, 2 * LBO_R, 128), ahi2 = smem_desc(shi, 2 * LBO_R, 128);
      const uint64_t bbase = smem_desc(sB1, 128, 256);
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const uint32_t dq = tmem + (uint32_t)(192 * qq);
#pragma unroll
        for (int J = 0; J < 8; ++J) {
          const bool lo = (J >> 2) & 1;
          const int row = 128 * qq - (J & 1) - kTile * ((J >> 1) & 1) + kShift;
#pragma unroll
          for (int i = 0; i < g1_count(J); ++i) {
            const int f = g1_first(J, i), g = g1_second(J, i);
            const uint64_t abase = (g - f == 2) ? (lo ? alo2 : ahi2) : (lo ? alo : ahi);
            const uint64_t ad = abase + (uint64_t)(((uint32_t)row * 16u + (uint32_t)f * LBO_R) >> 4);
            const uint64_t bd = bbase + (uint64_t)(((uint32_t)(g1_block(J) + i) * 2048u) >> 4);
            // J = 0 (hi) and J = 4 (lo) come first into their accumulators
            const bool first = (J & 3) == 0 && i == 0;
            mma_f16(dq + (lo ? 0u : 64u), ad, bd, idesc1, first ? 0u : 1u);
          }
        }
      }
      mma_commit(bar_g1);
    };
    // GEMM2 (one thread): out of cell layer kv - 1 from t(kv - 1), t(kv)
    auto issue_g2 = [&](int kv) {
      fence_after();
      const uint64_t a0 = smem_desc(sT + (uint32_t)(((kv - 1) & 1) * T_LAYER), LBO_T, 128);
      const uint64_t a1 = smem_desc(sT + (uint32_t)((kv & 1) * T_LAYER), LBO_T, 128);
      const uint64_t bbase = smem_desc(sB2, 128, 1024);
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const uint32_t dq = tmem + (uint32_t)(192 * qq) + 128u;
#pragma unroll
        for (int J = 0; J < 8; ++J) {
          const bool hi = (J >> 2) & 1;
          const int row = 128 * qq + (J & 1) + kTile * ((J >> 1) & 1);
          const uint32_t idesc2 = instr_desc(128, g2_n(J), FP16);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = (hi ? a1 : a0) + (uint64_t)(((uint32_t)row * 16u + (uint32_t)(2 * kk) * LBO_T) >> 4);
            const uint64_t bd = bbase + (uint64_t)(((uint32_t)g2_off(J) + (uint32_t)kk * 256u) >> 4);
            // the first MMA into each accumulator (J = 0, J = 4: N = 32) initialises it
            mma_f16(dq + (hi ? 32u : 0u), ad, bd, idesc2, ((J & 3) == 0 && kk == 0) ? 0u : 1u);
          }
        }
      }
      mma_commit(bar_g2);
    };

    // prologue: R(k0 - 1), R(k0); GEMM1 of vertex layer k0
    stage(k0 - 1);
    load_layer(k0);
    stage(k0);
    if (k0 + 1 <= k1) load_layer(k0 + 1);
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) issue_g1(k0);
    ++iss1;
    // iteration kv: out of cell layer kv - 2 into z, R(kv + 1), t(kv), then
    // GEMM2 of cell layer kv - 1 and GEMM1 of vertex layer kv + 1 back to back
    for (int kv = k0; kv <= k1; ++kv) {
      if (kv >= k0 + 2) {
        epi_load(kv - 2);
        if (mbar_wait(bar_g2, n2done & 1u)) ++n2done;
        else bad = true;
        fence_after();
        if (!__any_sync(0xffffffffu, bad)) epi_finish(kv - 2);
      }
      if (kv + 1 <= k1) {
        stage(kv + 1);
        if (kv + 2 <= k1) load_layer(kv + 2);
      }
      if (mbar_wait(bar_g1, n1done & 1u)) ++n1done;
      else bad = true;
      fence_after();
      if (!__any_sync(0xffffffffu, bad)) {
        const float slo = sc[(kv - 1) & 3], shi = sc[kv & 3];
        const float sg = fminf(slo, shi);
        if (tid == 0) sc[4 + (kv & 3)] = sg;
        const bool live = vtx_xy && kv >= 1 && kv <= nc - 1;
        const float flo = live ? sg / slo : 0.f, fhi = live ? sg / shi : 0.f;
        uint8_t* T8 = smem + OFF_T + (uint32_t)((kv & 1) * T_LAYER) + (uint32_t)m * 16u;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float a[16], b[16];
          const uint32_t col = (uint32_t)(32 * h + 16 * hh);
          tmem_ld16x2(tq + col, tq + 64 + col, a, b);
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            uint4 w;
            w.x = pack2<FP16>(a[8 * g + 0] * flo + b[8 * g + 0] * fhi, a[8 * g + 1] * flo + b[8 * g + 1] * fhi);
            w.y = pack2<FP16>(a[8 * g + 2] * flo + b[8 * g + 2] * fhi, a[8 * g + 3] * flo + b[8 * g + 3] * fhi);
            w.z = pack2<FP16>(a[8 * g + 4] * flo + b[8 * g + 4] * fhi, a[8 * g + 5] * flo + b[8 * g + 5] * fhi);
            w.w = pack2<FP16>(a[8 * g + 6] * flo + b[8 * g + 6] * fhi, a[8 * g + 7] * flo + b[8 * g + 7] * fhi);
            const uint32_t slice = (uint32_t)(4 * h + 2 * hh + g);
            *reinterpret_cast<uint4*>(T8 + slice * LBO_T) = w;
          }
        }
      }
      fence_async_smem();
      fence_before();
      if (agree()) break;
      if (tid == 0) {
        if (kv >= k0 + 1) issue_g2(kv);
        if (kv + 1 <= k1) issue_g1(kv + 1);
      }
      if (kv >= k0 + 1) ++iss2;
      if (kv + 1 <= k1) ++iss1;
    }
    if (bad) break;
    // out of the last cell layer of the chunk
    epi_load(k1 - 1);
    if (mbar_wait(bar_g2, n2done & 1u)) ++n2done;
    else bad = true;
    fence_after();
    if (agree()) break;
    epi_finish(k1 - 1);
    fence_before();
    __syncthreads();   // TMEM and the rings are free for the next item
  }
  if (bad) {
    // a wait gave up (every thread agreed): record it, wait (bounded) for the
    // products still outstanding (they may read the rings and write TMEM),
    // then free TMEM
    if (tid == 0) atomicExch(A.status, kTimeout);
    if (iss1 > n1done) mbar_wait(bar_g1, n1done & 1u);
    if (iss2 > n2done) mbar_wait(bar_g2, n2done & 1u);
    fence_before();
    __syncthreads();
  }
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_tc_cell_smoother_f16(CellArgs A) {
  pdl_start();
  cell_smoother_body<true>(A);
}
__global__ void __launch_bounds__(kThreads, 1) k_tc_cell_smoother_bf16(CellArgs A) {
  pdl_start();
  cell_smoother_body<false>(A);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// patch-local index of the edge at slot `slot` of the cell at offset o (each
// component -1 or 0) from the patch's vertex, or -1 if the patch does not
// hold it
static int patch_local(int slot, const int o[3]) {
  const int d = slot_d(slot);
  int p[3];
  for (int e = 0; e < 3; ++e) p[e] = 2 * (o[e] + 1) + slot_par(slot, e);
  return (int)Box{{4, 4, 4}}.index(d, p[0], p[1], p[2]);
}

std::vector<uint8_t> tc_cell_image(const std::vector<double>& W, bool fp16) {
  if (W.size() != (size_t)108 * 60) throw std::invalid_argument("tc_cell_image: W must be 108 x 60");
  double mx = 0.0;
  for (double v : W) mx = std::fmax(mx, std::fabs(v));
  const double sw = mx > 0 ? std::exp2(-std::ceil(std::log2(mx))) : 1.0;
  std::vector<uint8_t> img(kImgTotal, 0);
  auto put = [&](uint8_t* base, int row, int k, int K, double v) {
    uint16_t bits;
    if (fp16) {
      __half hv = __double2half(v);
      std::memcpy(&bits, &hv, 2);
    } else {
      __nv_bfloat16 bv = __double2bfloat16(v);
      std::memcpy(&bits, &bv, 2);
    }
    std::memcpy(base + core_off(row, k, K), &bits, 2);
  };
  // value of W'_o at position p, column c (0 when the neighbour does not hold it)
  auto wval = [&](int J, int p, int c) -> double {
    if (p >= 24 || c >= 60) return 0.0;
    const int s = pos_slot(p);
    if (slot_zero_mask(s) & J) return 0.0;
    const int o[3] = {(J & 1) ? -1 : 0, (J & 2) ? -1 : 0, (J & 4) ? -1 : 0};
    const int l = patch_local(s, o);
    if (l < 0) throw std::logic_error("tc_cell_image: slot map");
    return W[(size_t)l * 60 + c] * sw;
  };
  // GEMM1: per neighbour J and MMA i a 64 x 16 K-major block (rows = t
  // component, K = the 16 positions of the MMA's two K-slices)
  for (int J = 0; J < 8; ++J)
    for (int i = 0; i < g1_count(J); ++i) {
      uint8_t* blk = img.data() + (size_t)(g1_block(J) + i) * 2048;
      const int sl[2] = {g1_first(J, i), g1_second(J, i)};
      for (int c = 0; c < 64; ++c)
        for (int k = 0; k < 16; ++k) {
          const int slice = sl[k >> 3];
          const int p = 8 * slice + (k & 7);
          // the second of two MMAs repeats S1, which the first already covers
          const double v = (i == 1 && slice == 1) ? 0.0 : wval(J, p, c);
          put(blk, c, k, 16, v);
        }
    }
  // GEMM2: per neighbour J (offset +1 where bit set) an N x 64 K-major block
  // (rows = output position, K = t component); W'_{-o} has the masks of J
  for (int J = 0; J < 8; ++J) {
    uint8_t* blk = img.data() + kG1Bytes + g2_off(J);
    for (int p = 0; p < g2_n(J); ++p)
      for (int c = 0; c < 64; ++c) put(blk, p, c, 64, wval(J, p, c));
  }
  const float inv = (float)(1.0 / (sw * sw));
  std::memcpy(img.data() + kImgBytes, &inv, sizeof(float));
  return img;
}

cudaError_t prepare_tc_cell() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_cell_smoother_f16, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_cell_smoother_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  return e;
}

// chunk length along z that balances items over the SMs: each item costs
// its layers plus about two layers of pipeline fill
static int choose_zlen(int nc, int ncol, int R, int sm) {
  int best = nc;
  double best_t = 1e300;
  for (int zl = 1; zl <= nc; ++zl) {
    const int nzc = (nc + zl - 1) / zl;
    const long long items = (long long)ncol * ncol * nzc * R;
    const long long waves = (items + sm - 1) / sm;
    const double t = (double)waves * (zl + 2);
    if (t < best_t) {
      best_t = t;
      best = zl;
    }
  }
  return best;
}

void launch_tc_cell_smoother(cudaStream_t s, int sm, int n, const void* img, bool fp16, const float* AinvT,
                             double eta, const float* r, float* z, int* status, int R, int zlen) {
  const int nc = n / 2;
  if (nc < 2) return;
  CellArgs a;
  a.n = n;
  a.nc = nc;
  a.ncol = (nc + kOwn - 1) / kOwn;
  a.zlen = zlen > 0 ? (zlen < nc ? zlen : nc) : choose_zlen(nc, a.ncol, R, sm);
  a.nzc = (nc + a.zlen - 1) / a.zlen;
  a.items = a.ncol * a.ncol * a.nzc * R;
  a.eta = (float)eta;
  a.img = (const uint8_t*)img;
  a.AinvT = AinvT;
  a.r = r;
  a.z = z;
  a.status = status;
  const int grid = a.items < sm ? a.items : sm;
  if (fp16) launch_pdl(k_tc_cell_smoother_f16, grid, kThreads, kSmem, s, a);
  else launch_pdl(k_tc_cell_smoother_bf16, grid, kThreads, kSmem, s, a);
}

int tc_cell_image_bytes() { return kImgTotal; }

}  // namespace ndmg
