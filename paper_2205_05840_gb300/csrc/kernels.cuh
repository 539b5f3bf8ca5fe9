// Launchers of the CUDA-core kernels (kernels.cu) and the tensor-core
// vertex-patch kernel (tc_patch.cu).
#pragma once
#include "ndmg_internal.h"

namespace ndmg {

template <typename T>
void launch_stencil(cudaStream_t s, int sm, int n, double cK, double cM, const T* u, const T* g, T* y);
template <typename T>
void launch_stencil_simple(cudaStream_t s, int sm, int n, double cK, double cM, const T* u, const T* g, T* y);
template <typename T>
cudaError_t prepare_stencil();
template <typename T>
void launch_restrict(cudaStream_t s, int sm, int nf, const T* rf, T* gc);
template <typename T>
void launch_prolong_add(cudaStream_t s, int sm, int nf, const T* zc, T* zf);
template <typename T>
void launch_bubble(cudaStream_t s, int sm, int n, const T* Ainv, double eta, const T* r, T* z);
template <typename T>
cudaError_t prepare_vertex_dense();
template <typename T>
void launch_vertex_dense(cudaStream_t s, int sm, int n, const T* D, double eta, const T* r, T* z);
template <typename T>
void launch_coarse(cudaStream_t s, int N0, const double* Ainv, const T* g, T* z);
int reduction_blocks(int sm);
template <typename T>
void launch_dot2(cudaStream_t s, int sm, int64_t N, const T* x, const T* y, const T* x2, const T* y2,
                 double* partial, double* out);
template <typename T>
void launch_axpby(cudaStream_t s, int sm, int64_t N, double a, const T* x, double b, T* y);
template <typename T>
void launch_cg_update(cudaStream_t s, int sm, int64_t N, double a, const T* p, const T* q, T* u, T* r);
void launch_to_f32(cudaStream_t s, int sm, int64_t N, double sc, const double* src, float* dst);
void launch_add_f32(cudaStream_t s, int sm, int64_t N, double sc, const float* src, double* dst);
void launch_from_f32(cudaStream_t s, int sm, int64_t N, double sc, const float* src, double* dst);

}  // namespace ndmg
