// Tensor-core (tcgen05) vertex-patch solves of the mixed-precision smoother.
#pragma once
#include "ndmg_internal.h"

namespace ndmg {

// Build the device image of the Gram factor W (108x60, W W^t = J_V A_V^{-1}
// J_V^t) in the layout the tensor-core kernel reads (bf16 or fp16).
cudaError_t upload_tc_operand(void** dst, const std::vector<double>& W, bool fp16);
// Largest eigenvalue of A_p W~ W~^t for the rounded operand W~ of W (1 for
// the exact factor); the smoother loses its stability as it grows.
double tc_operand_spectral_max(const double* W, const std::vector<double>& Ap, bool fp16);
// Most the library accepts.  The value grows with the patch's conditioning,
// ~ alpha / (beta h^2), and depends on the bit patterns of the rounded factor
// as well: bf16 operands give 13 at alpha / (beta h^2) = 2.3e5 and 23 at
// 4.1e5 on 64^3 vertex patches, 4.8 and 7.3 at the same ratios on 32^3 and
// 128^3 (14 at 9.2e5 on 128^3); fp16 operands stay below 15 up to 2.5e7.  A
// bf16 solve with 23 at 4.1e5 diverged, one with 13 at 2.3e5 converged.
constexpr double kTcSpectralMax = 16.0;
// Opt in to the kernel's dynamic shared memory.
cudaError_t prepare_tc_patch();
// z += eta * (sum_T J_T A_T^{-1} J_T^t r + sum_V J_V A_V^{-1} J_V^t r) on
// level n (eq. (Preconditioner P); float r, z; R right-hand sides; AinvT the
// 6x6 interior-space inverse, row-major); on a device-side timeout the
// kernel writes a nonzero code to *status and adds nothing.  Persistent grid
// of at most 3 CTAs per SM (sm: the device's SM count).
void launch_tc_smoother(cudaStream_t s, int sm, int n, const void* Wimg, bool fp16, const float* AinvT, double eta,
                        const float* r, float* z, int* status, int R);
// Coefficient per hexahedron: device images of the Gram factors of ngroups
// vertex-patch groups (W: ngroups x 108 x 60), the per-brick group lists
// (off: bricks + 1 offsets; grp, mask: 4 words of row bits per entry) for the
// vertex groups vgid (vertex-family order), and the smoother with them
// (Atab: 36 floats per interior-space group, bub_gid per coarse element).
std::vector<uint8_t> tc_images(const std::vector<double>& W, int ngroups, bool fp16);
void tc_brick_groups(int n, const std::vector<int>& vgid, std::vector<int>* off, std::vector<int>* grp,
                     std::vector<uint32_t>* mask);
void launch_tc_smoother_field(cudaStream_t s, int n, const void* imgs, bool fp16, const float* Atab,
                              const int* bub_gid, const int* goff, const int* ggrp, const uint4* gmask, double eta,
                              const float* r, float* z, int* status, int R);

}  // namespace ndmg
