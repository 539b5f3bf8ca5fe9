// Floating-point conversions on the integer pipe.  GB300's FP64 pipe runs
// about 2 FMA per clock per SM (1/64 of the FP32 rate) and the FP64 <-> FP32
// conversion instructions share it, so the FP64 vector kernels form these
// conversions from the bit patterns instead.  Every function here is plain
// integer arithmetic on the IEEE-754 encodings; the header also compiles as
// host C++ (g++ or nvcc's host pass), which is how the library's CPU tests
// check each function bit for bit against the IEEE conversions.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define NDMG_HD __host__ __device__ __forceinline__
#else
#define NDMG_HD inline
#endif

namespace ndmg {

NDMG_HD unsigned long long bits_of(double x) {
#if defined(__CUDA_ARCH__)
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}

NDMG_HD double double_of(unsigned long long b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}

NDMG_HD uint32_t bits_of(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}

NDMG_HD float float_of(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}

// leading zero bits of a nonzero 64-bit word
NDMG_HD int clz64(unsigned long long a) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)a);
#else
  return __builtin_clzll(a);
#endif
}

// float -> double: exact for normal floats, subnormals flush to signed zero,
// infinities and NaN keep their class
NDMG_HD double f2d_bits(float f) {
  const uint32_t b = bits_of(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  const unsigned long long sgn = (unsigned long long)(b >> 31) << 63;
  const unsigned long long ed = e == 0xFFu ? 0x7FFull : (unsigned long long)(e + 896u);  // 1023 - 127
  const unsigned long long bits =
      e == 0u ? sgn : (sgn | (ed << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29));
  return double_of(bits);
}

// Power-of-two scales (the residual scaling of the mixed PCG).  A scale s
// is passed as its binary exponent k, s = 2^k; pow2_exponent(0) is a large
// negative k and pow2_exponent of an infinity or NaN a large positive one, so
// that the two functions below return signed zeros, respectively
// infinities, for them.
constexpr int kPow2Zero = -4096;
constexpr int kPow2Inf = 4096;

// binary exponent of s, which must be 0, a power of two, an infinity or NaN
NDMG_HD int pow2_exponent(double s) {
  const int e = (int)((bits_of(s) >> 52) & 0x7FF);
  return e == 0 ? kPow2Zero : (e == 0x7FF ? kPow2Inf : e - 1023);
}

// f 2^k as a double (exact; f subnormal gives a signed zero; a result outside
// the normal double range flushes to signed zero below and is an infinity
// above; f infinite or NaN keeps its class)
NDMG_HD double f2d_pow2(float f, int k) {
  const uint32_t b = bits_of(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  const unsigned long long sgn = (unsigned long long)(b >> 31) << 63;
  const unsigned long long frac = (unsigned long long)(b & 0x7FFFFFu) << 29;
  if (e == 0xFFu) return double_of(sgn | (0x7FFull << 52) | frac);
  const int ed = (int)e + 896 + k;
  if (e == 0u || ed <= 0) return double_of(sgn);
  if (ed >= 0x7FF) return double_of(sgn | (0x7FFull << 52));
  return double_of(sgn | ((unsigned long long)ed << 52) | frac);
}

// x 2^k rounded to the nearest float, ties to even (the IEEE conversion of
// the exact product), except that a result below the smallest normal float
// flushes to signed zero; overflow gives an infinity, NaN stays NaN
NDMG_HD float d2f_pow2(double x, int k) {
  const unsigned long long b = bits_of(x);
  const uint32_t sgn = (uint32_t)(b >> 32) & 0x80000000u;
  const int ed = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;  // 52 fraction bits
  if (ed == 0x7FF) return float_of(sgn | 0x7F800000u | (m ? 0x400000u : 0u));
  if (ed == 0) return float_of(sgn);                     // zero (and double subnormals)
  unsigned long long hi = m >> 29;                       // 23 fraction bits kept
  const unsigned long long rest = m & 0x1FFFFFFFull;     // 29 bits rounded away
  hi += (rest > 0x10000000ull || (rest == 0x10000000ull && (hi & 1ull))) ? 1ull : 0ull;
  int ef = ed - 896 + k;                                 // ed - 1023 + 127 + k
  if (hi >> 23) {                                        // the rounding carried out of the fraction
    hi = 0ull;
    ++ef;
  }
  if (ef <= 0) return float_of(sgn);
  if (ef >= 0xFF) return float_of(sgn | 0x7F800000u);
  return float_of(sgn | ((uint32_t)ef << 23) | (uint32_t)hi);
}

// v 2^s truncated toward zero to an int64 (the fixed point of the FP64
// stencil; requires |v| 2^s < 2^63, zero and subnormal v give 0)
NDMG_HD long long to_fixed(double v, int s) {
  const long long b = (long long)bits_of(v);
  const int e = (int)((b >> 52) & 0x7FF);
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
  const int sh = e - 1075 + s;  // v 2^s = m 2^sh
  long long r = sh >= 0 ? (long long)((unsigned long long)m << sh) : (sh > -63 ? (m >> -sh) : 0LL);
  r = e == 0 ? 0LL : r;         // zero and subnormals
  return b < 0 ? -r : r;
}

// int64 -> double rounded to nearest (ties to even): normalise |x| so that
// its leading one is bit 63, keep 53 bits, round on the 11 bits below,
// assemble sign / exponent / fraction
NDMG_HD double fixed_to_double(long long x) {
  if (x == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)x & 0x8000000000000000ull;
  unsigned long long a = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
  const int lz = clz64(a);
  a <<= lz;                                     // leading one at bit 63
  unsigned long long m = a >> 11;               // 53 significant bits
  const unsigned long long rest = a & 0x7FFull;  // the 11 bits rounded away
  m += (rest > 0x400ull || (rest == 0x400ull && (m & 1ull))) ? 1ull : 0ull;
  unsigned long long e = (unsigned long long)(1086 - lz);  // 1023 + 63 - lz
  if (m >> 53) {                                // rounding carried into bit 53
    m >>= 1;
    ++e;
  }
  return double_of(sgn | (e << 52) | (m & 0xFFFFFFFFFFFFFull));
}

}  // namespace ndmg
