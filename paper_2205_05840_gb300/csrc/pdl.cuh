// Programmatic dependent launch for the kernels of the V-cycle path.
//
// Consecutive kernels of a V-cycle depend on each other, and on the small
// levels a kernel does a few microseconds of work; the gap between the end of
// one kernel and the start of the next would be a large part of the time.
// Every kernel launched through launch_pdl may begin (its CTAs become
// resident) once all CTAs of the previous kernel in the stream have started;
// its first statement, pdl_start, lets the next kernel do the same and then
// waits until the previous kernel has completed and its memory is visible.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace ndmg {

__device__ __forceinline__ void pdl_start() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace ndmg
