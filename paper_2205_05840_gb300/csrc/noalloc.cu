// Inner product that allocates nothing (ndmg_dot_noalloc, see include/ndmg.h).
//
// Callers that cannot allocate device memory -- code running under an
// allocator that must own every device byte of the process, or code where a
// cudaMalloc (which may synchronise the device) is not acceptable, or code
// that cannot create a handle because ndmg_create allocates all level
// workspaces -- still need the library's FP64 reductions.  This entry point
// runs the same two-stage reduction as ndmg_dot, but its partial sums live in
// a file-scope device array of fixed size instead of a handle workspace.
#include <cstdio>
#include <mutex>

#include <cuda.h>

#include "ndmg_internal.h"

namespace ndmg {
namespace {

constexpr int kChunk = 16384;        // elements per block of the first stage
constexpr int kMaxChunks = 4096;     // => at most 67,108,864 elements
constexpr int kThreads = 256;

// partial sums of the first stage, then the result in slot kMaxChunks.
// Every GPU that loads this library holds these 32 KB until the process ends.
static __device__ __align__(256) double g_dot_scratch[kMaxChunks + 32];

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < kThreads / 32 ? ws[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;  // valid in thread 0
}

// block b sums x[i] * y[i] over its chunk [b * kChunk, (b + 1) * kChunk)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dot_chunks(const T* __restrict__ x, const T* __restrict__ y, int64_t n,
                                                         double* __restrict__ partial) {
  const int64_t lo = (int64_t)blockIdx.x * kChunk;
  const int64_t hi = lo + kChunk < n ? lo + kChunk : n;
  double v = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) v += (double)x[i] * (double)y[i];
  v = block_sum(v);
  if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kThreads) k_dot_finish(const double* __restrict__ partial, int nchunks,
                                                         double* __restrict__ result) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nchunks; b += kThreads) v += partial[b];
  v = block_sum(v);
  if (threadIdx.x == 0) *result = v;
}

// device address of g_dot_scratch, looked up once per device and CUDA
// context: a cudaDeviceReset (or a non-primary context on the same device)
// loads the module again, possibly at another address, so the cache is keyed
// by the id of the context current at the call (driver entry points fetched
// through the runtime, so the library needs no link against libcuda)
constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Cached {
  unsigned long long ctx_id = 0;  // 0: not looked up yet (driver context ids start at 1)
  double* addr = nullptr;
};
Cached g_addr[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// id of the context current on this thread (after the runtime made one current)
cudaError_t current_context_id(unsigned long long* id) {
  if (!g_ctx_current || !g_ctx_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
    g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  return g_ctx_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  // no context current yet on this thread, a new context, or a first call:
  // look the address up (the lookup makes the device's primary context
  // current), then record which context it belongs to
  if (current_context_id(&id) != cudaSuccess || g_addr[dev].ctx_id != id || !g_addr[dev].addr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dot_scratch);
    if (e == cudaSuccess) e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    g_addr[dev].addr = static_cast<double*>(p);
    g_addr[dev].ctx_id = id;
  }
  *out = g_addr[dev].addr;
  return cudaSuccess;
}

}  // namespace
}  // namespace ndmg

extern "C" int ndmg_dot_noalloc(int32_t dtype, const void* x, const void* y, int64_t n, double* out, void* stream) {
  using namespace ndmg;
  if (!out || n < 0 || (dtype != NDMG_F64 && dtype != NDMG_F32)) return NDMG_INVALID_ARG;
  if (n > (int64_t)kChunk * kMaxChunks) {
    std::fprintf(stderr, "ndmg_dot_noalloc: n = %lld exceeds the static scratch limit of %lld elements\n",
                 (long long)n, (long long)kChunk * kMaxChunks);
    return NDMG_INVALID_ARG;
  }
  if (n == 0) {
    *out = 0.0;
    return NDMG_OK;
  }
  if (!x || !y || ((uintptr_t)x & 15u) || ((uintptr_t)y & 15u)) return NDMG_INVALID_ARG;
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return NDMG_CUDA_ERROR;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nchunks = (int)((n + kChunk - 1) / kChunk);
  // every partial slot the finish kernel reads is written by the first kernel,
  // so nothing needs clearing between calls
  if (dtype == NDMG_F64)
    k_dot_chunks<double><<<nchunks, kThreads, 0, s>>>((const double*)x, (const double*)y, n, scratch);
  else
    k_dot_chunks<float><<<nchunks, kThreads, 0, s>>>((const float*)x, (const float*)y, n, scratch);
  k_dot_finish<<<1, kThreads, 0, s>>>(scratch, nchunks, scratch + kMaxChunks);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, scratch + kMaxChunks, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? NDMG_OK : NDMG_CUDA_ERROR;
}
