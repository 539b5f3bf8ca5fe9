// Tensor-core vertex-patch kernel (tcgen05): not built yet; ndmg_create
// rejects the mixed precision modes until it is.
#include "tc_patch.cuh"

namespace ndmg {

cudaError_t upload_tc_operand(void**, const std::vector<double>&, bool) { return cudaErrorNotSupported; }
cudaError_t prepare_tc_patch() { return cudaErrorNotSupported; }
void launch_tc_patch(cudaStream_t, int, int, const void*, bool, double, const float*, float*, int*) {}

}  // namespace ndmg
