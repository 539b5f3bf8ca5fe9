// Cell-owned tensor-core smoother (tc_cell.cu): the vertex-space solves of
// eq. (Preconditioner P) as shifted-row GEMMs on tcgen05, one writer per edge.
#pragma once
#include "ndmg_internal.h"

namespace ndmg {

// Device image (fp16 or bf16) of the Gram factor W (108 x 60, patch-local
// order) in the per-neighbour blocks the kernel reads, scaled by a power of
// two (max |W| <= 1), followed by the float 1 / scale^2.
std::vector<uint8_t> tc_cell_image(const std::vector<double>& W, bool fp16);
int tc_cell_image_bytes();
// Opt in to the kernel's dynamic shared memory.
cudaError_t prepare_tc_cell();
// z += eta * (sum_T J_T A_T^{-1} J_T^t r + sum_V J_V W W^t J_V^t r) on level
// n (float r, z; R right-hand sides; AinvT the 6 x 6 interior-space inverse;
// sm: CTAs of the persistent grid; zlen: cell layers per work item, 0 = the
// built-in choice).  On a device-side timeout the kernel writes a nonzero
// code to *status and stops adding (z may then hold a partial update).
void launch_tc_cell_smoother(cudaStream_t s, int sm, int n, const void* img, bool fp16, const float* AinvT,
                             double eta, const float* r, float* z, int* status, int R, int zlen = 0);

}  // namespace ndmg
