// Tensor-core (tcgen05) vertex-patch solves of the mixed-precision smoother.
#pragma once
#include "ndmg_internal.h"

namespace ndmg {

// Build the device image of the Gram factor W (108x60, W W^t = J_V A_V^{-1}
// J_V^t) in the layout the tensor-core kernel reads (bf16 or fp16).
cudaError_t upload_tc_operand(void** dst, const std::vector<double>& W, bool fp16);
// Opt in to the kernel's dynamic shared memory.
cudaError_t prepare_tc_patch();
// z += eta * (sum_T J_T A_T^{-1} J_T^t r + sum_V J_V A_V^{-1} J_V^t r) on
// level n (eq. (Preconditioner P); float r, z; R right-hand sides; AinvT the
// 6x6 interior-space inverse, row-major); on a device-side timeout the
// kernel writes a nonzero code to *status and adds nothing.
void launch_tc_smoother(cudaStream_t s, int n, const void* Wimg, bool fp16, const float* AinvT, double eta,
                        const float* r, float* z, int* status, int R);

}  // namespace ndmg
