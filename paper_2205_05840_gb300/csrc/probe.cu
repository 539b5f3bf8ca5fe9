// Measured CUDA-core FMA rate (ndmg_probe_fma_rate, include/ndmg.h): the
// denominator of the roofline of the kernels bound by the FP64 or FP32 pipes
// (the CUDA-core patch solves of FP64 handles, the FP64 PCG updates).  Many
// warps each run independent chains of fused multiply-adds; the rate is the
// FMAs done over the time of the launch (CUDA events), as FLOP/s = 2 FMA/s.
#include "ndmg_internal.h"

namespace ndmg {
namespace {

constexpr int kChains = 8;     // independent FMA chains per thread (enough ILP for the pipe latency)
constexpr int kIters = 4096;   // FMAs per chain
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_rate(T a, T b, T* out) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 4
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == (T)12345.678) out[0] = s;   // never true for these inputs; keeps the chains alive
}

template <typename T>
cudaError_t rate(int sm, double* tflops) {
  T* out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(T));
  if (e != cudaSuccess) return e;
  const int grid = sm * 8;   // 64 warps per SM
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_rate<T><<<grid, kThreads>>>((T)0.999, (T)1e-4, out);   // warm-up
  cudaEventRecord(e0);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) k_fma_rate<T><<<grid, kThreads>>>((T)0.999, (T)1e-4, out);
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e == cudaSuccess) {
    const double fmas = (double)reps * grid * kThreads * kChains * kIters;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  }
  return e;
}

}  // namespace
}  // namespace ndmg

extern "C" int ndmg_probe_fma_rate(int32_t dtype, double* tflops) {
  if (!tflops || (dtype != NDMG_F64 && dtype != NDMG_F32)) return NDMG_INVALID_ARG;
  int dev = 0, sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return NDMG_CUDA_ERROR;
  const cudaError_t e = dtype == NDMG_F64 ? ndmg::rate<double>(sm, tflops) : ndmg::rate<float>(sm, tflops);
  return e == cudaSuccess ? NDMG_OK : NDMG_CUDA_ERROR;
}
