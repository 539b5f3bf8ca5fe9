// The smallest levels of the float V-cycle in one thread-block cluster
// (coarse_cycle.cu).
#pragma once
#include "ndmg_internal.h"

namespace ndmg {

constexpr int kCoarseMaxLevels = 3;   // levels above the coarsest handled by one launch
constexpr int kCoarseMaxN = 16;       // largest level size n handled

struct CoarseLevel {
  int n;
  double cK, cM;          // alpha h and beta h^3
  float *g, *z, *r;       // right-hand side, solution, residual workspace (R right-hand sides each)
  const float* W;         // 108 x 60 Gram factor (FP32, row-major)
  const float* AinvT;     // 6 x 6 interior-space inverse (FP32)
};

cudaError_t prepare_coarse_cycle();
// CTAs of the cluster, 0 if such a cluster cannot be resident on this device
int coarse_cycle_grid(int sm_count, int Kc);
// z_Kc = MG(Kc, g_Kc, 0, m) of Fig. 1 over levels lv[Kc] .. lv[1] and the
// coarsest level (g0, z0: N0 values per right-hand side, Ainv0 its inverse);
// z_Kc must be zero on entry.  status: the handle's status word (the kernel
// does nothing while it is nonzero).  grid: coarse_cycle_grid's value.
cudaError_t launch_coarse_cycle(cudaStream_t s, int grid, const CoarseLevel* lv, int Kc, int N0, const double* Ainv0,
                                float* g0, float* z0, double eta, int m, int R, int* status);

}  // namespace ndmg
