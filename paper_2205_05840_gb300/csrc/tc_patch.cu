// Smoother correction of eq. (Preconditioner P) with the vertex-space solves
// on the 5th-gen tensor cores (tcgen05, sm_103a):
//
//     z += eta * ( sum_T J_T A_T^{-1} J_T^t r  +  sum_V J_V A_V^{-1} J_V^t r ),
//
// with J_V A_V^{-1} J_V^t = W W^t, W the 108x60 Gram factor of the vertex
// space operator (identical for every patch: constant alpha, uniform grid).
// One kernel, k_tc_smoother.  A CTA takes a brick of 8 x 4 x 4 interior coarse
// vertices (one 128-row MMA tile; neighbouring rows are neighbouring vertices
// along x) and
//   1. stages r on the cells the brick's patches cover (row-wise cp.async,
//      zero fill outside the box = the boundary condition), split by the
//      parity of the cell coordinates so that neighbouring patches read
//      neighbouring words;
//   2. gathers the 128 patch vectors into A (128 x 112, bf16/fp16, K-major);
//   3. D = A W             (tcgen05.mma M=128 N=64  K=112, FP32 in TMEM);
//   4. A' = lowp(D)        (tcgen05.ld -> registers -> smem, over A);
//   5. D' = A' W^t         (tcgen05.mma M=128 N=112 K=64, FP32 in TMEM, over D);
//   6. adds the 108 outputs of every patch and the interior-space solves of
//      the coarse elements the brick owns into a shared-memory copy of the
//      region (over A'), and
//   7. adds that copy, times eta, to z with coalesced global reductions.
// Every patch is computed once; edges near a brick face receive the
// contributions of both bricks through the global reductions.
//
// Operand layout (SWIZZLE_NONE, K-major canonical layout): 8-row x 16-byte
// "core matrices" stored contiguously; core matrix (g, c) of an R x K
// operand (g = row / 8, c = k / 8) sits at byte (g * K/8 + c) * 128.
// Descriptor: leading byte offset (next core matrix along K) = 128, stride
// byte offset (next 8-row group) = K/8 * 128.
#include <cmath>
#include <cstring>
#include <type_traits>

#include "tc_patch.cuh"
#include "pdl.cuh"

namespace ndmg {
namespace {

constexpr int kBX = 8, kBY = 4, kBZ = 4;   // coarse vertices per brick
constexpr int kM = 128;                    // MMA rows = kBX * kBY * kBZ patches
static_assert(kBX * kBY * kBZ == kM, "one MMA tile per brick");
constexpr int kK1 = 112, kN1 = 64;         // A: 128 x 112, W: 112 x 64
constexpr int kK2 = 64, kN2 = 112;         // A': 128 x 64, W^t: 64 x 112
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 128;        // D: cols [0,64), then D': cols [0,112)

// staged region: cells [2V0 - 2, 2(V0 + B - 1) + 2] per axis, i.e. 2B + 2
// cells; per direction the along-axis extent counts segments (2B + 2) and
// the across extents count node lines (2B + 1)
constexpr int kCX = 2 * kBX + 2, kCY = 2 * kBY + 2, kCZ = 2 * kBZ + 2;
__host__ __device__ constexpr int dir_len(int d, int axis) {
  return (axis == 0 ? kCX : axis == 1 ? kCY : kCZ) - (axis == d ? 0 : 1);
}
__host__ __device__ constexpr int dir_size(int d) { return dir_len(d, 0) * dir_len(d, 1) * dir_len(d, 2); }
constexpr int kRegionAll = dir_size(0) + dir_size(1) + dir_size(2);

// octant (parity-split) layout of the staged region
__host__ __device__ constexpr int oct_len(int L, int par) { return (L + 1 - par) / 2; }
__host__ __device__ constexpr int oct_size(int d, int o) {
  return oct_len(dir_len(d, 0), o & 1) * oct_len(dir_len(d, 1), (o >> 1) & 1) * oct_len(dir_len(d, 2), (o >> 2) & 1);
}
__host__ __device__ constexpr int oct_base(int d, int o) {
  int base = 0;
  for (int q = 0; q < d; ++q) base += dir_size(q);
  for (int q = 0; q < o; ++q) base += oct_size(d, q);
  return base;
}
static_assert(oct_base(2, 7) + oct_size(2, 7) == kRegionAll, "octants tile the region");

__host__ __device__ constexpr int region_at_c(int d, int i, int j, int k) {
  const int o = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
  const int PI = oct_len(dir_len(d, 0), i & 1);
  const int PJ = PI * oct_len(dir_len(d, 1), j & 1);
  return oct_base(d, o) + (k >> 1) * PJ + (j >> 1) * PI + (i >> 1);
}

// The staged region in canonical order, one direction after another (i
// fastest): entry = octant-layout index | i << 13 | j << 18 | k << 22.  Both
// the staging of r and the flush into z walk it with all lanes busy.
struct RegionTable {
  uint32_t v[kRegionAll];
};
constexpr RegionTable make_region_table() {
  RegionTable t{};
  int q = 0;
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k < dir_len(d, 2); ++k)
      for (int j = 0; j < dir_len(d, 1); ++j)
        for (int i = 0; i < dir_len(d, 0); ++i)
          t.v[q++] = (uint32_t)region_at_c(d, i, j, k) | ((uint32_t)i << 13) | ((uint32_t)j << 18) | ((uint32_t)k << 22);
  return t;
}
static_assert(kRegionAll < (1 << 13) && kCX <= 32 && kCY <= 16 && kCZ <= 16, "region table fields");
__device__ const RegionTable kRegionTab = make_region_table();

// Calls f(table entry, global offset within one right-hand side, edge is
// interior) for every element of the direction-D part of the region (the
// entry holds the octant-layout index in bits 0-12 and the region
// coordinates i, j, k in bits 13-17, 18-21, 22-25).  Region
// element (i, j, k) of direction D is the edge at global coordinates
// 2 V0 + (i, j, k) - (2 along D, 1 across).
template <int D, typename F>
__device__ __forceinline__ void walk_region(int n, int VX, int VY, int VZ, int tid, F&& f) {
  constexpr int q0 = D == 0 ? 0 : (D == 1 ? dir_size(0) : dir_size(0) + dir_size(1));
  const uint32_t n1 = n - 1, N3 = (uint32_t)n * n1 * n1;
  const int gi0 = 2 * VX - (D == 0 ? 2 : 1), gj0 = 2 * VY - (D == 1 ? 2 : 1), gk0 = 2 * VZ - (D == 2 ? 2 : 1);
  // all table entries of this thread first: the copies / reductions below are
  // ordered memory operations, so a load inside the loop would wait a full
  // round trip per element
  constexpr int kIt = (dir_size(D) + kThreads - 1) / kThreads;
  uint32_t ent[kIt];
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int q = tid + it * kThreads;
    ent[it] = q < dir_size(D) ? __ldg(&kRegionTab.v[q0 + q]) : 0u;
  }
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    if (tid + it * kThreads >= dir_size(D)) break;
    const uint32_t e = ent[it];
    const int gi = gi0 + (int)((e >> 13) & 31u), gj = gj0 + (int)((e >> 18) & 15u), gk = gk0 + (int)(e >> 22);
    bool in;
    uint32_t off;
    if (D == 0) {
      in = (unsigned)gi < (unsigned)n && (unsigned)(gj - 1) < n1 && (unsigned)(gk - 1) < n1;
      off = ((uint32_t)(gk - 1) * n1 + (uint32_t)(gj - 1)) * n + (uint32_t)gi;
    } else if (D == 1) {
      in = (unsigned)(gi - 1) < n1 && (unsigned)gj < (unsigned)n && (unsigned)(gk - 1) < n1;
      off = N3 + ((uint32_t)(gk - 1) * n + (uint32_t)gj) * n1 + (uint32_t)(gi - 1);
    } else {
      in = (unsigned)(gi - 1) < n1 && (unsigned)(gj - 1) < n1 && (unsigned)gk < (unsigned)n;
      off = 2u * N3 + ((uint32_t)gk * n1 + (uint32_t)(gj - 1)) * n1 + (uint32_t)(gi - 1);
    }
    f(e, off, in);
  }
}

// shared memory: A' aliases A (A is dead once the first MMA completed), and
// the region accumulator aliases A' once both products are complete
constexpr int OFF_A = 0;
constexpr int OFF_B1 = OFF_A + kM * kK1 * 2;  // W images, contiguous
constexpr int OFF_B2 = OFF_B1 + kN1 * kK1 * 2;
constexpr int OFF_R = OFF_B2 + kN2 * kK2 * 2;
constexpr int OFF_BAR = OFF_R + ((kRegionAll * 4 + 15) / 16) * 16;
constexpr int OFF_TM = OFF_BAR + 16;
constexpr int OFF_RED = OFF_TM + 16;
constexpr int OFF_AT = OFF_RED + 48;          // A_T^{-1} (6 x 6, FP32); red: 8 warp maxima + 1 flag
constexpr int kSmem = OFF_AT + 36 * 4;
static_assert(kRegionAll * 4 <= kM * kK1 * 2, "accumulator fits in the A operand");
static_assert(OFF_BAR % 8 == 0, "mbarrier alignment");
static_assert(3 * (kSmem + 1024) <= 228 * 1024, "three CTAs per SM (228 KB, 1 KB reserved per CTA)");

// coefficient field (one W per group of patches): A is kept for every group
// of the brick, so A' and the accumulator get their own space
constexpr int OFF_A2F = (kSmem + 127) / 128 * 128;
constexpr int OFF_ACCF = OFF_A2F + kM * kK2 * 2;
constexpr int kSmemF = OFF_ACCF + ((kRegionAll * 4 + 15) / 16) * 16;
static_assert(2 * (kSmemF + 1024) <= 228 * 1024, "two CTAs per SM (228 KB, 1 KB reserved per CTA)");

constexpr int kImgBytes = (kN1 * kK1 + kN2 * kK2) * 2;  // both W images
constexpr int kImgStride = kImgBytes + 16;               // one image and its scale
constexpr int kLoBytes = kN2 * kK2 * 2;                   // low-order part of the second W image
constexpr int kFieldImgStride = kImgStride + kLoBytes;    // one group's image and its low-order part
static_assert(kLoBytes <= ((kRegionAll * 4 + 15) / 16) * 16, "the low-order image fits the region buffer");
static_assert(OFF_B2 - OFF_B1 == kN1 * kK1 * 2 && OFF_R - OFF_B1 == kImgBytes, "W images are one block");
constexpr int kTimeout = 1;                              // status code

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) in a K-major no-swizzle operand of width K
__host__ __device__ constexpr int core_off(int row, int k, int K) {
  return ((row >> 3) * (K >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the tcgen05 family
  return d;                // base offset 0, absolute LBO mode, no swizzle
}

// instruction descriptor, kind::f16: D f32, A/B bf16 (or f16), both K-major
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, bool fp16) {
  return (1u << 4) | ((fp16 ? 0u : 1u) << 7) | ((fp16 ? 0u : 1u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: gives up after 2^20 polls or ~5e8 cycles (~0.25 s)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (int it = 0; it < (1 << 20); ++it) {
    if (mbar_try(bar, parity)) return true;
    if (clock64() - t0 > 500000000LL) break;
  }
  return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 4-byte asynchronous copy global -> shared; src_bytes = 0 writes a zero
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per thread)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

template <bool FP16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if constexpr (FP16) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
}

// Patch-local edge l in [0,108): the canonical numbering of the 4x4x4 box
// of cells around the vertex (x: 4 segments x 3 x 3 node lines, then y, then
// z).  Its region coordinates for brick-relative vertex (a,b,c) are the box
// coordinates + 2(a,b,c) - (0 along the edge, 1 across); everything below
// constant-folds for a literal l.
__host__ __device__ constexpr int local_dir(int l) { return l < 36 ? 0 : (l < 72 ? 1 : 2); }
__host__ __device__ constexpr int local_ri(int l) { return l < 36 ? l % 4 : (l < 72 ? (l - 36) % 3 : (l - 72) % 3); }
__host__ __device__ constexpr int local_rj(int l) {
  return l < 36 ? (l / 4) % 3 : (l < 72 ? ((l - 36) / 3) % 4 : ((l - 72) / 3) % 3);
}
__host__ __device__ constexpr int local_rk(int l) { return l < 36 ? l / 12 : (l < 72 ? (l - 36) / 12 : (l - 72) / 9); }

// staged-region index of patch-local edge l of the patch at (a,b,c): the
// patch moves by 2 cells per vertex, i.e. by one entry of its octant
__device__ __forceinline__ int patch_elem(int l, int a, int b, int c) {
  const int d = local_dir(l), i = local_ri(l), j = local_rj(l), k = local_rk(l);
  const int PI = oct_len(dir_len(d, 0), i & 1);
  const int PJ = PI * oct_len(dir_len(d, 1), j & 1);
  return region_at_c(d, i, j, k) + c * PJ + b * PI + a;
}

// 7 chunks of 8 patch-local edges from chunk CH0 on, rounded to bf16/fp16 and
// stored as 16-byte rows of the K-major operand A
template <int CH0, bool FP16>
__device__ __forceinline__ void gather_chunks(const float* R, uint8_t* A, int p, int a, int b, int c, bool live,
                                              float rscale) {
#pragma unroll
  for (int ch = CH0; ch < CH0 + 7; ++ch) {
    float v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int l = ch * 8 + t;
      v[t] = (live && l < 108) ? R[patch_elem(l, a, b, c)] * rscale : 0.f;
    }
    uint4 w;
    w.x = pack2<FP16>(v[0], v[1]);
    w.y = pack2<FP16>(v[2], v[3]);
    w.z = pack2<FP16>(v[4], v[5]);
    w.w = pack2<FP16>(v[6], v[7]);
    *reinterpret_cast<uint4*>(A + core_off(p, ch * 8, kK1)) = w;
  }
}

// Octant index of interior edge w of the coarse element E = V0 - 1 + (ei,
// ej, ek): its edge of direction dw = w / 2 has segment 2 E_dw + (w & 1) and
// nodes 2 E + 1 across, i.e. region coordinates 2 (ei, ej, ek) + (w & 1 along,
// 0 across); the parities, hence the octant, are fixed by w
__device__ __forceinline__ int bubble_elem(int w, int ei, int ej, int ek) {
  const int dw = w >> 1, s = w & 1;
  const int ri = 2 * ei + (dw == 0 ? s : 0), rj = 2 * ej + (dw == 1 ? s : 0), rk = 2 * ek + (dw == 2 ? s : 0);
  const int o = (dw == 0 ? s : 0) | ((dw == 1 ? s : 0) << 1) | ((dw == 2 ? s : 0) << 2);
  const int PI = oct_len(dir_len(dw, 0), ri & 1);
  const int PJ = PI * oct_len(dir_len(dw, 1), rj & 1);
  return oct_base(dw, o) + (rk >> 1) * PJ + (rj >> 1) * PI + (ri >> 1);
}

// 16 columns [C0, C0 + 16) of D' for this thread's patch row, added into the
// accumulator at the patch's edges (compile-time patch-local indices)
template <int C0>
__device__ __forceinline__ void scatter16(uint32_t taddr, float* acc, int a, int b, int c, float sc) {
  float v[16];
  tmem_ld16(taddr + C0, v);
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    if (C0 + t < 108) atomicAdd(acc + patch_elem(C0 + t, a, b, c), v[t] * sc);
  }
}

// D = A W: M = 128, N = 64, K = 112 (one elected thread)
template <bool FP16>
__device__ __forceinline__ void issue_mma1(uint32_t tmem, uint32_t a0, uint32_t b0, uint32_t bar) {
  const uint32_t idesc = instr_desc(kM, kN1, FP16);
#pragma unroll
  for (int kk = 0; kk < kK1 / 16; ++kk)
    mma_f16(tmem, smem_desc(a0 + kk * 256, 128, (kK1 / 8) * 128), smem_desc(b0 + kk * 256, 128, (kK1 / 8) * 128),
            idesc, kk > 0);
  mma_commit(bar);
}

// D' = A' W^t: M = 128, N = 112, K = 64 (one elected thread)
template <bool FP16>
__device__ __forceinline__ void issue_mma2(uint32_t tmem, uint32_t a0, uint32_t b0, uint32_t bar) {
  const uint32_t idesc = instr_desc(kM, kN2, FP16);
#pragma unroll
  for (int kk = 0; kk < kK2 / 16; ++kk)
    mma_f16(tmem, smem_desc(a0 + kk * 256, 128, (kK2 / 8) * 128), smem_desc(b0 + kk * 256, 128, (kK2 / 8) * 128),
            idesc, kk > 0);
  mma_commit(bar);
}

// D' = A' (W_hi + W_lo)^t: the product above, then the same with the
// low-order image at b0lo into the same accumulator (one elected thread)
template <bool FP16>
__device__ __forceinline__ void issue_mma2_split(uint32_t tmem, uint32_t a0, uint32_t b0, uint32_t b0lo, uint32_t bar) {
  const uint32_t idesc = instr_desc(kM, kN2, FP16);
#pragma unroll
  for (int kk = 0; kk < kK2 / 16; ++kk)
    mma_f16(tmem, smem_desc(a0 + kk * 256, 128, (kK2 / 8) * 128), smem_desc(b0 + kk * 256, 128, (kK2 / 8) * 128),
            idesc, kk > 0);
#pragma unroll
  for (int kk = 0; kk < kK2 / 16; ++kk)
    mma_f16(tmem, smem_desc(a0 + kk * 256, 128, (kK2 / 8) * 128), smem_desc(b0lo + kk * 256, 128, (kK2 / 8) * 128),
            idesc, true);
  mma_commit(bar);
}

// A' = low-precision copy of D (8 warps: lane quadrant x column half)
template <bool FP16>
__device__ __forceinline__ void convert_d(uint32_t tmem, uint8_t* A2, int warp, int lane) {
  const int p = (warp & 3) * 32 + lane;
  const int cb0 = (warp >> 2) * 32;
#pragma unroll 1
  for (int cb = cb0; cb < cb0 + 32; cb += 16) {
    float v[16];
    tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + cb, v);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint4 w;
      w.x = pack2<FP16>(v[8 * h + 0], v[8 * h + 1]);
      w.y = pack2<FP16>(v[8 * h + 2], v[8 * h + 3]);
      w.z = pack2<FP16>(v[8 * h + 4], v[8 * h + 5]);
      w.w = pack2<FP16>(v[8 * h + 6], v[8 * h + 7]);
      *reinterpret_cast<uint4*>(A2 + core_off(p, cb + 8 * h, kK2)) = w;
    }
  }
}

// rows of D' (this warp's lane quadrant, its column half) added into the
// region accumulator, scaled by scl (0 for rows that add nothing)
__device__ __forceinline__ void scatter_rows(uint32_t tmem, float* acc, int warp, int lane, float scl) {
  const int prow = (warp & 3) * 32 + lane;
  const int a = prow % kBX, b = (prow / kBX) % kBY, c = prow / (kBX * kBY);
  const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  // tcgen05.ld is warp-collective: every lane loads
  if (warp < 4) {
    scatter16<0>(taddr, acc, a, b, c, scl);
    scatter16<16>(taddr, acc, a, b, c, scl);
    scatter16<32>(taddr, acc, a, b, c, scl);
    scatter16<48>(taddr, acc, a, b, c, scl);
  } else {
    scatter16<64>(taddr, acc, a, b, c, scl);
    scatter16<80>(taddr, acc, a, b, c, scl);
    scatter16<96>(taddr, acc, a, b, c, scl);
  }
}

template <bool FP16>
__global__ void __launch_bounds__(kThreads, 3)
    k_tc_smoother(int n, const uint8_t* __restrict__ img, const float* __restrict__ AinvT, float eta,
                  const float* __restrict__ r, float* __restrict__ z, int* __restrict__ status, int R) {
  // the next kernel may start its own set-up now; this kernel's set-up
  // (TMEM, barriers, the W images and A_T^{-1}) reads nothing the previous
  // kernel writes, so it runs before the wait for that kernel
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nv = n / 2 - 1;
  const int nbx = (nv + kBX - 1) / kBX, nby = (nv + kBY - 1) / kBY, nbz = (nv + kBZ - 1) / kBZ;
  const int nbr = nbx * nby * nbz;
  const uint32_t n1 = n - 1, N3 = (uint32_t)n * n1 * n1;  // < 2^31 (checked on the host)

  float* R_ = reinterpret_cast<float*>(smem + OFF_R);
  float* ACC = reinterpret_cast<float*>(smem + OFF_A);  // region accumulator, over A' once D' is complete
  float* At = reinterpret_cast<float*>(smem + OFF_AT);
  const uint32_t bar0 = smem_u32(smem + OFF_BAR), bar1 = bar0 + 8;
  uint32_t* tm_slot = reinterpret_cast<uint32_t*>(smem + OFF_TM);
  float* red = reinterpret_cast<float*>(smem + OFF_RED);

  // ---- set-up, once per CTA: TMEM, barriers, both W images, A_T^{-1} ---------
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tm_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar1), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 36) At[tid] = __ldg(AinvT + tid);
  {
    const uint4* src = reinterpret_cast<const uint4*>(img);
    const uint32_t wbase = smem_u32(smem + OFF_B1);
    for (int q = tid; q < kImgBytes / 16; q += kThreads)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(wbase + 16u * q), "l"(src + q) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  const float wscale = __ldg(reinterpret_cast<const float*>(img + kImgBytes));  // 1 / s_w^2
  asm volatile("griddepcontrol.wait;" ::: "memory");  // r, z and the status word of the previous kernels
  // a CTA of an earlier launch gave up on a wait: do nothing until the host
  // has read and cleared the status word
  const bool quiet = *reinterpret_cast<volatile int*>(status) != 0;
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tm_slot;

  // ---- one brick of one right-hand side per pass -----------------------------
  uint32_t parity = 0;
  for (int w = quiet ? R * nbr : blockIdx.x; w < R * nbr; w += gridDim.x, parity ^= 1u) {
    const int rhs = w / nbr, brick = w - rhs * nbr;
    const int bx = brick % nbx, by = (brick / nbx) % nby, bz = brick / (nbx * nby);
    const int VX = 1 + bx * kBX, VY = 1 + by * kBY, VZ = 1 + bz * kBZ;  // first vertex of the brick
    const float* rr = r + (int64_t)rhs * 3 * N3;
    float* zr = z + (int64_t)rhs * 3 * N3;

    // ---- 1. stage r on the region ---------------------------------------------
    {
      const uint32_t rbase = smem_u32(R_);
      auto stage = [&](uint32_t e, uint32_t off, bool in) {
        cp_async4(rbase + 4u * (e & 8191u), rr + (in ? off : 0u), in ? 4u : 0u);
      };
      walk_region<0>(n, VX, VY, VZ, tid, stage);
      walk_region<1>(n, VX, VY, VZ, tid, stage);
      walk_region<2>(n, VX, VY, VZ, tid, stage);
      asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();

    // fp16 operands: scale r by a power of two so that max |r| <= 1 on the region
    float rscale = 1.f;
    if constexpr (FP16) {
      float amax = 0.f;
      for (int q = tid; q < kRegionAll; q += kThreads) amax = fmaxf(amax, fabsf(R_[q]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if (lane == 0) red[warp] = amax;
      __syncthreads();
      float m = 0.f;
#pragma unroll
      for (int q = 0; q < kThreads / 32; ++q) m = fmaxf(m, red[q]);
      if (m > 0.f) rscale = exp2f(-ceilf(log2f(m)));
    }

    // ---- 2. gather the patch vectors into A (two threads per row) --------------
    {
      const int p = tid & (kM - 1), half = tid >> 7;
      const int a = p % kBX, b = (p / kBX) % kBY, c = p / (kBX * kBY);
      const bool live = VX + a <= nv && VY + b <= nv && VZ + c <= nv;
      uint8_t* A = smem + OFF_A;
      if (half == 0)
        gather_chunks<0, FP16>(R_, A, p, a, b, c, live, rscale);
      else
        gather_chunks<7, FP16>(R_, A, p, a, b, c, live, rscale);
    }
    // interior spaces of the coarse elements the brick owns: E in [V0-1, V1-1]
    // per axis, plus element nv on the last brick of an axis (its last vertex
    // is nv); the 6 interior edges of E are row t = 2d + (segment parity).
    // Solved now, while r is staged, and added into the accumulator later.
    constexpr int kBubMax = ((kBX + 1) * (kBY + 1) * (kBZ + 1) * 6 + kThreads - 1) / kThreads;
    int bub_at[kBubMax];
    float bub_v[kBubMax];
    {
      const int ex1 = VX + kBX - 1 >= nv ? nv : VX + kBX - 2;
      const int ey1 = VY + kBY - 1 >= nv ? nv : VY + kBY - 2;
      const int ez1 = VZ + kBZ - 1 >= nv ? nv : VZ + kBZ - 2;
      const int mx = ex1 - VX + 2, my = ey1 - VY + 2, mz = ez1 - VZ + 2;
#pragma unroll
      for (int w = 0; w < kBubMax; ++w) {
        const int q = tid + w * kThreads;
        bub_at[w] = -1;
        bub_v[w] = 0.f;
        if (q < mx * my * mz * 6) {
          const int t = q % 6, e = q / 6;
          const int ei = e % mx, ej = (e / mx) % my, ek = e / (mx * my);  // E - (V0 - 1)
          float sum = 0.f;
          int it = 0;
#pragma unroll
          for (int u = 0; u < 6; ++u) {
            const int ix = bubble_elem(u, ei, ej, ek);
            sum += At[t * 6 + u] * R_[ix];
            if (u == t) it = ix;
          }
          bub_at[w] = it;
          bub_v[w] = sum;
        }
      }
    }
    fence_async_smem();
    __syncthreads();  // A is complete and r is no longer read

    // ---- 3. D = A W; the low-order image of W^t into the region buffer ------------
    if (tid == 0) {
      fence_after();
      issue_mma1<FP16>(tmem, smem_u32(smem + OFF_A), smem_u32(smem + OFF_B1), bar0);
    }
    {
      const uint4* src = reinterpret_cast<const uint4*>(img + kImgStride);
      const uint32_t lbase = smem_u32(smem + OFF_R);
      for (int q = tid; q < kLoBytes / 16; q += kThreads)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(lbase + 16u * q), "l"(src + q) : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    bool ok = mbar_wait(bar0, parity);
    fence_after();

    // ---- 4. A' = low-precision copy of D (8 warps: lane quadrant x column half)
    if (ok) convert_d<FP16>(tmem, smem + OFF_A, warp, lane);
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // the low-order image landed
    fence_async_smem();
    fence_before();
    __syncthreads();

    // ---- 5. D' = A' W^t, written over D -----------------------------------------
    // (issued only when thread 0 saw the first product complete; red[8] tells
    // every thread whether it was)
    if (tid == 0) {
      red[8] = ok ? 1.f : 0.f;
      if (ok) {
        fence_after();
        issue_mma2_split<FP16>(tmem, smem_u32(smem + OFF_A), smem_u32(smem + OFF_B2), smem_u32(smem + OFF_R), bar1);
      }
    }
    if (ok) ok = mbar_wait(bar1, parity);
    fence_after();
    // the CTA goes on only if every thread saw both products complete
    ok = __syncthreads_and(ok) != 0;
    if (!ok) {
      // a wait gave up: the products issued so far may still be reading A', W
      // and writing TMEM.  Record the timeout, touch no shared memory, wait
      // (again bounded) for those products, free TMEM and return.
      if (tid == 0) atomicExch(status, kTimeout);
      mbar_wait(bar0, parity);
      if (red[8] != 0.f) mbar_wait(bar1, parity);
      fence_before();
      __syncthreads();
      if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
      }
      return;
    }
    // A' has been read by the tensor cores: its space becomes the accumulator
    for (int q = tid; q < kRegionAll; q += kThreads) ACC[q] = 0.f;
    __syncthreads();

    // ---- 6. accumulate: patch outputs (rows of D') and interior-space solves ----
    {
      const int prow = (warp & 3) * 32 + lane;
      const int a = prow % kBX, b = (prow / kBX) % kBY, c = prow / (kBX * kBY);
      const bool live = VX + a <= nv && VY + b <= nv && VZ + c <= nv;
      scatter_rows(tmem, ACC, warp, lane, live ? wscale / rscale : 0.f);  // live rows add
    }
    // the interior-space solves formed before the products
#pragma unroll
    for (int w = 0; w < kBubMax; ++w)
      if (bub_at[w] >= 0) atomicAdd(ACC + bub_at[w], bub_v[w]);
    fence_before();
    __syncthreads();

    // ---- 7. z += eta * accumulator ---------------------------------------------
    {
      auto flush = [&](uint32_t e, uint32_t off, bool in) {
        if (in) atomicAdd(zr + off, eta * ACC[e & 8191u]);
      };
      walk_region<0>(n, VX, VY, VZ, tid, flush);
      walk_region<1>(n, VX, VY, VZ, tid, flush);
      walk_region<2>(n, VX, VY, VZ, tid, flush);
    }
    // the next pass rewrites R, A (= the accumulator) and TMEM
    fence_before();
    __syncthreads();
    fence_after();
  }
  if (quiet) asm volatile("cp.async.wait_group 0;" ::: "memory");  // the W images copied for nothing
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// The same smoother for a curl-curl coefficient constant per hexahedron:
// the brick's patches fall into groups with their own Gram factors W_g
// (host lists per brick: groups[off[b] .. off[b+1]) with 128-bit row masks).
// A is gathered once; for each group the kernel loads W_g, forms D = A W_g
// and D' = lowp(D) W_g^t, and adds only the rows of that group.  The interior
// solves use the 6x6 inverse of each coarse element's group (Atab, 36 floats
// per group, bub_gid per coarse element).
template <bool FP16>
__global__ void __launch_bounds__(kThreads, 2)
    k_tc_smoother_field(int n, const uint8_t* __restrict__ imgs, const float* __restrict__ Atab,
                        const int* __restrict__ bub_gid, const int* __restrict__ goff, const int* __restrict__ ggrp,
                        const uint4* __restrict__ gmask, float eta, const float* __restrict__ r,
                        float* __restrict__ z, int* __restrict__ status) {
  pdl_start();
  extern __shared__ __align__(128) uint8_t smem[];
  if (*reinterpret_cast<volatile int*>(status) != 0) return;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nv = n / 2 - 1, nc = n / 2;
  const int nbx = (nv + kBX - 1) / kBX, nby = (nv + kBY - 1) / kBY, nbz = (nv + kBZ - 1) / kBZ;
  const int nbr = nbx * nby * nbz;
  const int rhs = blockIdx.x / nbr;
  const int brick = blockIdx.x - rhs * nbr;
  const int bx = brick % nbx, by = (brick / nbx) % nby, bz = brick / (nbx * nby);
  const int VX = 1 + bx * kBX, VY = 1 + by * kBY, VZ = 1 + bz * kBZ;
  const uint32_t n1 = n - 1, N3 = (uint32_t)n * n1 * n1;
  r += (int64_t)rhs * 3 * N3;
  z += (int64_t)rhs * 3 * N3;

  float* R = reinterpret_cast<float*>(smem + OFF_R);
  float* ACC = reinterpret_cast<float*>(smem + OFF_ACCF);
  uint8_t* A2 = smem + OFF_A2F;
  const uint32_t bar0 = smem_u32(smem + OFF_BAR), bar1 = bar0 + 8;
  uint32_t* tm_slot = reinterpret_cast<uint32_t*>(smem + OFF_TM);
  float* red = reinterpret_cast<float*>(smem + OFF_RED);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tm_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar1), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    const uint32_t rbase = smem_u32(R);
    auto stage = [&](uint32_t e, uint32_t off, bool in) {
      cp_async4(rbase + 4u * (e & 8191u), r + (in ? off : 0u), in ? 4u : 0u);
    };
    walk_region<0>(n, VX, VY, VZ, tid, stage);
    walk_region<1>(n, VX, VY, VZ, tid, stage);
    walk_region<2>(n, VX, VY, VZ, tid, stage);
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
  }
  for (int q = tid; q < kRegionAll; q += kThreads) ACC[q] = 0.f;
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tm_slot;

  float rscale = 1.f;
  if constexpr (FP16) {
    float amax = 0.f;
    for (int q = tid; q < kRegionAll; q += kThreads) amax = fmaxf(amax, fabsf(R[q]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) red[warp] = amax;
    __syncthreads();
    float m = 0.f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) m = fmaxf(m, red[w]);
    if (m > 0.f) rscale = exp2f(-ceilf(log2f(m)));
  }

  {
    const int p = tid & (kM - 1), half = tid >> 7;
    const int a = p % kBX, b = (p / kBX) % kBY, c = p / (kBX * kBY);
    const bool live = VX + a <= nv && VY + b <= nv && VZ + c <= nv;
    uint8_t* A = smem + OFF_A;
    if (half == 0)
      gather_chunks<0, FP16>(R, A, p, a, b, c, live, rscale);
    else
      gather_chunks<7, FP16>(R, A, p, a, b, c, live, rscale);
  }

  // interior spaces of the coarse elements the brick owns (see k_tc_smoother),
  // solved while r is staged; the region buffer then takes each group's
  // low-order W image
  {
    const int ex1 = VX + kBX - 1 >= nv ? nv : VX + kBX - 2;
    const int ey1 = VY + kBY - 1 >= nv ? nv : VY + kBY - 2;
    const int ez1 = VZ + kBZ - 1 >= nv ? nv : VZ + kBZ - 2;
    const int mx = ex1 - VX + 2, my = ey1 - VY + 2, mz = ez1 - VZ + 2;
    auto item = [&](int t, int ei, int ej, int ek) {
      const int EI = VX - 1 + ei, EJ = VY - 1 + ej, EK = VZ - 1 + ek;  // coarse element
      const float* At = Atab + 36 * (size_t)__ldg(bub_gid + ((size_t)EK * nc + EJ) * nc + EI);
      int idx[6];
#pragma unroll
      for (int w = 0; w < 6; ++w) idx[w] = bubble_elem(w, ei, ej, ek);
      float s = 0.f;
      int it = idx[0];
#pragma unroll
      for (int w = 0; w < 6; ++w) {
        s += __ldg(At + t * 6 + w) * R[idx[w]];
        if (w == t) it = idx[w];
      }
      atomicAdd(ACC + it, s);
    };
    for (int q = tid; q < mx * my * mz * 6; q += kThreads) {
      const int e = q / 6;
      item(q % 6, e % mx, (e / mx) % my, e / (mx * my));
    }
  }
  __syncthreads();  // r is no longer read

  // ---- one pass per group of patches in the brick ---------------------------
  const int e0 = __ldg(goff + brick), e1 = __ldg(goff + brick + 1);
  const int prow = (warp & 3) * 32 + lane;
  const int pa = prow % kBX, pb = (prow / kBX) % kBY, pc = prow / (kBX * kBY);
  const bool live = VX + pa <= nv && VY + pb <= nv && VZ + pc <= nv;
  bool ok = true;
  const uint32_t wbase = smem_u32(smem + OFF_B1);
  uint32_t last_parity = 0;
  for (int e = e0; e < e1 && ok; ++e) {
    const uint32_t parity = (uint32_t)(e - e0) & 1u;
    last_parity = parity;
    const uint8_t* img = imgs + (size_t)__ldg(ggrp + e) * kFieldImgStride;
    const uint4 mk = __ldg(gmask + e);
    const uint32_t word = prow < 32 ? mk.x : prow < 64 ? mk.y : prow < 96 ? mk.z : mk.w;
    const bool mine = live && ((word >> (prow & 31)) & 1u);
    // W_g into B1 / B2 (the previous group's products have completed)
    const uint4* src = reinterpret_cast<const uint4*>(img);
    for (int q = tid; q < kImgBytes / 16; q += kThreads)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(wbase + 16u * q), "l"(src + q) : "memory");
    {
      const uint4* lsrc = reinterpret_cast<const uint4*>(img + kImgStride);
      const uint32_t lbase = smem_u32(smem + OFF_R);
      for (int q = tid; q < kLoBytes / 16; q += kThreads)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(lbase + 16u * q), "l"(lsrc + q) : "memory");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    const float wscale = __ldg(reinterpret_cast<const float*>(img + kImgBytes));
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      issue_mma1<FP16>(tmem, smem_u32(smem + OFF_A), wbase, bar0);
    }
    bool okg = mbar_wait(bar0, parity);
    fence_after();
    if (okg) convert_d<FP16>(tmem, A2, warp, lane);
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      red[8] = okg ? 1.f : 0.f;  // whether the second product of this group was issued
      if (okg) {
        fence_after();
        issue_mma2_split<FP16>(tmem, smem_u32(A2), smem_u32(smem + OFF_B2), smem_u32(smem + OFF_R), bar1);
      }
    }
    if (okg) okg = mbar_wait(bar1, parity);
    fence_after();
    ok = __syncthreads_and(okg) != 0;
    if (ok) scatter_rows(tmem, ACC, warp, lane, mine ? wscale / rscale : 0.f);
    fence_before();
    __syncthreads();  // TMEM, A' and B are free for the next group
    fence_after();
  }
  if (!ok) {
    // a wait gave up: record it, wait (bounded) for the products of the last
    // group, which may still read A, A', W and write TMEM, free TMEM, return
    if (tid == 0) atomicExch(status, kTimeout);
    mbar_wait(bar0, last_parity);
    if (red[8] != 0.f) mbar_wait(bar1, last_parity);
    fence_before();
    __syncthreads();
    if (warp == 0) {
      fence_after();
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
    return;
  }

  fence_before();
  __syncthreads();

  if (ok) {
    auto flush = [&](uint32_t e, uint32_t off, bool in) {
      if (in) atomicAdd(z + off, eta * ACC[e & 8191u]);
    };
    walk_region<0>(n, VX, VY, VZ, tid, flush);
    walk_region<1>(n, VX, VY, VZ, tid, flush);
    walk_region<2>(n, VX, VY, VZ, tid, flush);
  }
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

// image of one Gram factor W (108 x 60 row-major) at img (kImgStride bytes):
// both operand layouts, scaled by a power of two so that max |W| <= 1, then
// the float 1 / scale^2
// The operand images of W: B1 for D = A W (W scaled by sw, max |W sw| in
// (1/2, 1]) and B2 for D' = A' W^t (scaled by sw2 = 2^12 sw, so that the
// low-order part below stays clear of the subnormal range); the float after
// both is 1 / (sw sw2).  lo (optional): B2's low-order part, W sw2 minus its
// rounding, in the same format and layout.  Rounding W in the second product
// moves the smoother's output out of the vertex space and costs V-cycles;
// the first product's rounding only perturbs coefficients inside it, so only
// the second product gets the low-order part.
static void tc_image(const double* Wp, bool fp16, uint8_t* img, uint8_t* lo = nullptr) {
  const std::vector<double> W(Wp, Wp + 108 * 60);
  double mx = 0.0;
  for (double v : W) mx = std::fmax(mx, std::fabs(v));
  const double sw = mx > 0 ? std::exp2(-std::ceil(std::log2(mx))) : 1.0;
  const double sw2 = sw * 4096.0;
  auto round_to = [&](double v) {
    return fp16 ? (double)__half2float(__double2half(v)) : (double)__bfloat162float(__double2bfloat16(v));
  };
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
  std::memset(img, 0, kImgStride);
  if (lo) std::memset(lo, 0, kLoBytes);
  uint8_t* b1 = img;                           // B1[n][k] = W[k][n]: N = 64, K = 112
  uint8_t* b2 = img + kN1 * kK1 * 2;           // B2[n][k] = W[n][k]: N = 112, K = 64
  for (int l = 0; l < 108; ++l)
    for (int c = 0; c < 60; ++c) {
      const double w = W[(size_t)l * 60 + c];
      put(b1, c, l, kK1, w * sw);
      put(b2, l, c, kK2, w * sw2);
      if (lo) put(lo, l, c, kK2, w * sw2 - round_to(w * sw2));
    }
  const float inv = (float)(1.0 / (sw * sw2));
  std::memcpy(img + kImgBytes, &inv, sizeof(float));
}

// Largest eigenvalue of A_p W~ W~^t with W~ the operand image's rounded W
// (scale included): 1 for the exact Gram factor (A_p W W^t is a projection),
// larger as the rounding meets ill-conditioned patches.  Power iteration on
// A_p^{1/2} W~ W~^t A_p^{1/2} (symmetric PSD) through y = W~ W~^t A_p x.
double tc_operand_spectral_max(const double* Wp, const std::vector<double>& Ap, bool fp16) {
  std::vector<uint8_t> img(kImgStride, 0);
  tc_image(Wp, fp16, img.data());
  float inv = 0.f;
  std::memcpy(&inv, img.data() + kImgBytes, sizeof(float));
  std::vector<double> Wr((size_t)108 * 60);
  // B2[l][c] = W[l][c] sw2 rounded, with sw2 = 4096 sw and inv = 1 / (sw sw2):
  // the rounding of the first product's operand, the one the kernel keeps
  const double unscale = std::sqrt((double)inv / 4096.0);  // 1 / sw2
  const uint8_t* b2 = img.data() + kN1 * kK1 * 2;
  for (int l = 0; l < 108; ++l)
    for (int c = 0; c < 60; ++c) {
      uint16_t bits;
      std::memcpy(&bits, b2 + core_off(l, c, kK2), 2);
      double v;
      if (fp16) {
        __half hv;
        std::memcpy(&hv, &bits, 2);
        v = (double)__half2float(hv);
      } else {
        __nv_bfloat16 bv;
        std::memcpy(&bv, &bits, 2);
        v = (double)__bfloat162float(bv);
      }
      Wr[(size_t)l * 60 + c] = v * unscale;
    }
  std::vector<double> x(108, 1.0), ax(108), t(60), y(108);
  for (int l = 0; l < 108; ++l) x[l] = 1.0 + 0.01 * l;  // not orthogonal to the top eigenvector
  double lam = 0.0;
  for (int it = 0; it < 60; ++it) {
    for (int a = 0; a < 108; ++a) {
      double s = 0.0;
      for (int b = 0; b < 108; ++b) s += Ap[(size_t)a * 108 + b] * x[b];
      ax[a] = s;
    }
    for (int c = 0; c < 60; ++c) {
      double s = 0.0;
      for (int l = 0; l < 108; ++l) s += Wr[(size_t)l * 60 + c] * ax[l];
      t[c] = s;
    }
    double num = 0.0, den = 0.0;
    for (int l = 0; l < 108; ++l) {
      double s = 0.0;
      for (int c = 0; c < 60; ++c) s += Wr[(size_t)l * 60 + c] * t[c];
      y[l] = s;
      den += x[l] * ax[l];
    }
    for (int c = 0; c < 60; ++c) num += t[c] * t[c];  // x^t A W~ W~^t A x
    lam = den > 0 ? num / den : 0.0;                   // Rayleigh quotient in the A_p inner product
    double nrm = 0.0;
    for (int l = 0; l < 108; ++l) nrm += y[l] * y[l];
    nrm = std::sqrt(nrm);
    if (!(nrm > 0)) break;
    for (int l = 0; l < 108; ++l) x[l] = y[l] / nrm;
  }
  return lam;
}

cudaError_t upload_tc_operand(void** dst, const std::vector<double>& W, bool fp16) {
  std::vector<uint8_t> img(kImgStride + kLoBytes, 0);  // the image, then B2's low-order part
  tc_image(W.data(), fp16, img.data(), img.data() + kImgStride);
  if (!*dst) {
    cudaError_t e = cudaMalloc(dst, img.size());
    if (e != cudaSuccess) return e;
  }
  return cudaMemcpy(*dst, img.data(), img.size(), cudaMemcpyHostToDevice);
}

cudaError_t prepare_tc_patch() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_smoother<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_smoother<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_smoother_field<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemF);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_smoother_field<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemF);
  return e;
}

std::vector<uint8_t> tc_images(const std::vector<double>& W, int ngroups, bool fp16) {
  std::vector<uint8_t> out((size_t)ngroups * kFieldImgStride);
  for (int q = 0; q < ngroups; ++q) {
    uint8_t* img = out.data() + (size_t)q * kFieldImgStride;
    tc_image(W.data() + (size_t)q * 108 * 60, fp16, img, img + kImgStride);
  }
  return out;
}

void tc_brick_groups(int n, const std::vector<int>& vgid, std::vector<int>* off, std::vector<int>* grp,
                     std::vector<uint32_t>* mask) {
  const int nv = n / 2 - 1;
  const int nbx = (nv + kBX - 1) / kBX, nby = (nv + kBY - 1) / kBY, nbz = (nv + kBZ - 1) / kBZ;
  off->assign(1, 0);
  grp->clear();
  mask->clear();
  for (int bz = 0; bz < nbz; ++bz)
    for (int by = 0; by < nby; ++by)
      for (int bx = 0; bx < nbx; ++bx) {
        const size_t first = grp->size();
        for (int p = 0; p < kM; ++p) {
          const int vx = 1 + bx * kBX + p % kBX, vy = 1 + by * kBY + (p / kBX) % kBY, vz = 1 + bz * kBZ + p / (kBX * kBY);
          if (vx > nv || vy > nv || vz > nv) continue;
          const int g = vgid[((size_t)(vz - 1) * nv + (vy - 1)) * nv + (vx - 1)];
          size_t e = first;
          while (e < grp->size() && (*grp)[e] != g) ++e;
          if (e == grp->size()) {
            grp->push_back(g);
            mask->insert(mask->end(), 4, 0u);
          }
          (*mask)[4 * e + p / 32] |= 1u << (p % 32);
        }
        off->push_back((int)grp->size());
      }
}

void launch_tc_smoother_field(cudaStream_t s, int n, const void* imgs, bool fp16, const float* Atab,
                              const int* bub_gid, const int* goff, const int* ggrp, const uint4* gmask, double eta,
                              const float* r, float* z, int* status, int R) {
  const int nv = n / 2 - 1;
  if (nv < 1) return;
  const int grid = ((nv + kBX - 1) / kBX) * ((nv + kBY - 1) / kBY) * ((nv + kBZ - 1) / kBZ) * R;
  if (fp16)
    launch_pdl(k_tc_smoother_field<true>, grid, kThreads, kSmemF, s, n, (const uint8_t*)imgs, Atab, bub_gid, goff, ggrp,
                                                               gmask, (float)eta, r, z, status);
  else
    launch_pdl(k_tc_smoother_field<false>, grid, kThreads, kSmemF, s, n, (const uint8_t*)imgs, Atab, bub_gid, goff, ggrp,
                                                                gmask, (float)eta, r, z, status);
}

void launch_tc_smoother(cudaStream_t s, int sm, int n, const void* Wimg, bool fp16, const float* AinvT, double eta,
                        const float* r, float* z, int* status, int R) {
  const int nv = n / 2 - 1;
  if (nv < 1) return;
  // persistent: at most three CTAs per SM (the shared-memory limit), each
  // taking every grid-th brick of every right-hand side
  const int64_t work = (int64_t)((nv + kBX - 1) / kBX) * ((nv + kBY - 1) / kBY) * ((nv + kBZ - 1) / kBZ) * R;
  const int grid = (int)(work < 3LL * sm ? work : 3LL * sm);
  if (fp16)
    launch_pdl(k_tc_smoother<true>, grid, kThreads, kSmem, s, n, (const uint8_t*)Wimg, AinvT, (float)eta, r, z, status,
               R);
  else
    launch_pdl(k_tc_smoother<false>, grid, kThreads, kSmem, s, n, (const uint8_t*)Wimg, AinvT, (float)eta, r, z,
               status, R);
}


}  // namespace ndmg
