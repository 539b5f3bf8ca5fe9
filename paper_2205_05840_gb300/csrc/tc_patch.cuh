// Tensor-core (tcgen05) vertex-patch solves of the mixed-precision smoother.
#pragma once
#include "ndmg_internal.h"

namespace ndmg {

// Build the device image of the Gram factor W (108x60, W W^t = J_V A_V^{-1}
// J_V^t) in the layout the tensor-core kernel reads (bf16 or fp16).
cudaError_t upload_tc_operand(void** dst, const std::vector<double>& W, bool fp16);
// Opt in to the kernel's dynamic shared memory.
cudaError_t prepare_tc_patch();
// Floats of the per-patch output buffer y of one right-hand side on level n:
// 108 x (n/2 - 1)^3.
int64_t tc_patch_buffer_floats(int n);
// y[l][p] = (J_V A_V^{-1} J_V^t r)_l of every vertex patch p on level n
// (float r; R right-hand sides); on a device-side timeout the kernel writes a
// nonzero code to *status.
void launch_tc_patches(cudaStream_t s, int n, const void* Wimg, bool fp16, const float* r, float* y, int* status,
                       int R);
// z += eta * (sum_T J_T A_T^{-1} J_T^t r + sum of the patch outputs y of each
// edge), eq. (Preconditioner P), one thread per lattice point.
void launch_vertex_gather(cudaStream_t s, int n, const float* y, const float* AinvT, double eta, const float* r,
                          float* z, int R);

}  // namespace ndmg
