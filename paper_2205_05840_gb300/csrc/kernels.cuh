// Launchers of the CUDA-core kernels (kernels.cu).  R = right-hand sides in
// the batch; every right-hand side is a contiguous canonical vector.
#pragma once
#include "ndmg_internal.h"

namespace ndmg {

// y = g - (cK K + cM M) u, or (cK K + cM M) u when g is null (cK = alpha h,
// cM = beta h^3 for A_k).  For double vectors the operator runs in exact
// fixed point; umax is R words of device scratch for its scale, which the
// launch forms from u first unless umax_ready (then they hold max |u| bits
// already).  kz: planes per CTA along z (0 = the built-in choice; any value
// gives the same result).  pq (double apply only): room for pq_cap block
// partial sums per right-hand side; when the launch's blocks per right-hand
// side fit, it also leaves the partial sums of u.y there (layout of
// k_dot2) and returns their number per right-hand side, else it returns 0
// and writes none.
template <typename T>
int launch_stencil(cudaStream_t s, int sm, int n, double cK, double cM, const T* u, const T* g, T* y, int R,
                   unsigned long long* umax, int kz = 0, bool umax_ready = false, double* pq = nullptr,
                   int64_t pq_cap = 0);
template <typename T>
cudaError_t prepare_stencil();
// g_c = P^t r_f; with zc, also z_c = 0
template <typename T>
void launch_restrict(cudaStream_t s, int sm, int nf, const T* rf, T* gc, int R, T* zc = nullptr);
template <typename T>
void launch_prolong_add(cudaStream_t s, int sm, int nf, const T* zc, T* zf, int R);
template <typename T>
void launch_bubble(cudaStream_t s, int sm, int n, const T* Ainv, double eta, const T* r, T* z, int R);
template <typename T>
cudaError_t prepare_vertex_dense();
// small levels (at most 4096 vertex patches): interior and vertex-patch
// solves of eq. (Preconditioner P) in one launch, FP32 (D: the 108 x 108
// operator, Ainv: the 6 x 6 interior inverse), z += eta * M^{-1} r
bool smooth_direct_fits(int n);
cudaError_t prepare_smooth_direct();
void launch_smooth_direct(cudaStream_t s, int n, const float* D, const float* Ainv, double eta, const float* r,
                          float* z, int R);
template <typename T>
void launch_vertex_dense(cudaStream_t s, int sm, int n, const T* D, double eta, const T* r, T* z, int R);
// A lattice of box-shaped patches (see k_patch_dense in kernels.cu).
struct PatchFamily {
  int nloc;        // interior edges of one box
  int b[3];        // box extents in cells
  int np[3];       // patches per axis
  int p0[3];       // first patch index per axis
  int shift[3];    // box origin = stride * patch index - shift
  int stride = 2;  // cells between neighbouring patches
};
PatchFamily vertex_family(int n);
PatchFamily edge_family(int n, int d);
// subdomain size 4: the 4x4x4-cell subdomains (interior spaces, 108 edges)
// and the 8x8x8-cell vertex patches around their interior vertices (1176)
PatchFamily subdomain4_family(int n);
PatchFamily vertex4_family(int n);
// z += eta * W (W^t r_p) for every patch p of the family (W: nloc x nG
// row-major, WT: its transpose), batches of patches per CTA
template <typename T>
void launch_patch_gram(cudaStream_t s, int sm, int n, const PatchFamily& fam, int nG, const T* W, const T* WT,
                       double eta, const T* r, T* z, int R);
template <typename T>
cudaError_t prepare_patch_gram();
// entries of one dense nl x nl operator in device memory: FP32 operators
// plain; FP64 ones followed by their hi / lo float parts (the double-float
// kernel's operands)
template <typename T>
constexpr size_t dense_stride(int nl) {
  return sizeof(T) == 8 ? 2 * (size_t)nl * nl : (size_t)nl * nl;
}
// FP64 patch solves in the basis of the patch box's mirror symmetries
// (patch_sym.cu): build_patch_sym turns a dense nloc x nloc operator D of the
// family's box into the kernel's tables and block-diagonal factor (false:
// the box has no such structure; dropped: the largest off-block entry, which
// is rounding noise, relative to the largest entry); launch_patch_sym adds
// eta * D r_p into z for every patch p, and with Ainv (the 6 x 6 interior
// inverse) also the interior-space solves of every coarse element, in the
// same launch
bool build_patch_sym(const PatchFamily& fam, const double* D, std::vector<uint32_t>* blob, double* dropped);
cudaError_t prepare_patch_sym();
void launch_patch_sym(cudaStream_t s, int sm, int n, const PatchFamily& fam, const uint32_t* blob, int blob_words,
                      double eta, const double* r, double* z, int R, const double* Ainv = nullptr);
// the FP32 smoother (vertex patches in the same basis, FP32 block products,
// and the 6 x 6 interior solves Ainv) in one launch: z += eta * M^{-1} r;
// blob: the vertex operator's tables (stored padded to 16 bytes)
cudaError_t prepare_smooth_sym32();
void launch_smooth_sym32(cudaStream_t s, int n, const uint32_t* blob, int blob_words, const float* Ainv, double eta,
                         const float* r, float* z, int R);
// z += eta * D r_p for every patch p of the family; D: one operator in the
// dense_stride<T> layout (FP64: the double-float kernel)
template <typename T>
void launch_patch_dense(cudaStream_t s, int sm, int n, const PatchFamily& fam, const T* D, double eta, const T* r,
                        T* z, int R);
template <typename T>
void launch_coarse(cudaStream_t s, int N0, const double* Ainv, const T* g, T* z, int R);
// coefficient field: the operator with a coefficient per cell (acell, n^3;
// cK = h times the pencil factor), interior solves and patch solves with one
// operator per group, and the per-cell derivative -lambda^T K_T u
template <typename T>
cudaError_t prepare_stencil_field();
template <typename T>
void launch_stencil_field(cudaStream_t s, int sm, int n, double cK, double cM, const T* u, const T* g, T* y, int R,
                          const T* acell, int kz = 0);
template <typename T>
void launch_bubble_grouped(cudaStream_t s, int sm, int n, const T* Atab, const int* gid, double eta, const T* r, T* z,
                           int R);
int patch_group_size();
template <typename T>
cudaError_t prepare_patch_grouped();
template <typename T>
void launch_patch_grouped(cudaStream_t s, int sm, int n, const PatchFamily& fam, const T* Dtab, const int4* chunks,
                          int nchunks, const int* plist, double eta, const T* r, T* z, int R);
void launch_grad_cells(cudaStream_t s, int sm, int n, double h, const double* lam, const double* u, double* out,
                       int R);
// -lambda_r^T K u_r per right-hand side into out[2 r] in one fused pass (K
// the alpha-free curl-curl matrix, or sum_T acell_T K_T when acell is given)
void launch_grad_alpha_sum(cudaStream_t s, int sm, int n, double h, const double* lam, const double* u,
                           const double* acell, double* partial, double* out, int R);
int reduction_blocks(int sm);
// PCG scalars on the device from the block partial sums of one reduction
// (modes CgMode; flex: the preconditioned residual is sfrom * z32)
void launch_cg_scalars(cudaStream_t s, int mode, int nb, const double* partial, const CgScalars& S, bool flex,
                       int* status, int R);
// reductions that leave their block partial sums for launch_cg_scalars
template <typename T>
void launch_dot2_partial(cudaStream_t s, int sm, int64_t N, const T* x, const T* y, const T* x2, const T* y2,
                         double* partial, int R);
void launch_cg_update_rr_partial(cudaStream_t s, int sm, int64_t N, const double* alpha, const double* p,
                                 const double* q, double* u, double* r, const double* sto, float* g32,
                                 double* partial, int R);
// (umax0: optional words set to 0 for launch_axpby_zf)
void launch_dot2_zf_partial(cudaStream_t s, int sm, int64_t N, const double* x, const double* y, const float* z32,
                            double* partial, int R, unsigned long long* umax0 = nullptr);
template <typename T>
void launch_dot2(cudaStream_t s, int sm, int64_t N, const T* x, const T* y, const T* x2, const T* y2,
                 double* partial, double* out, int R);
template <typename T>
void launch_axpby(cudaStream_t s, int sm, int64_t N, const double* ab, const T* x, T* y, int R);
template <typename T>
void launch_axpby_scalar(cudaStream_t s, int sm, int64_t N, double a, const T* x, double b, T* y);
template <typename T>
void launch_cg_update(cudaStream_t s, int sm, int64_t N, const double* alpha, const T* p, const T* q, T* u, T* r,
                      int R);
// fused steps of the mixed flexible PCG (reductions: partials + finisher into
// out[2 rhs], like launch_dot2)
void launch_cg_update_rr(cudaStream_t s, int sm, int64_t N, const double* alpha, const double* p, const double* q,
                         double* u, double* r, const double* sto, float* g32, double* partial, double* out, int R);
// out[2 rhs + {0,1}] = x.z32, y.z32 (unscaled: the caller multiplies by the
// scale of z32)
void launch_dot2_zf(cudaStream_t s, int sm, int64_t N, const double* x, const double* y, const float* z32,
                    double* partial, double* out, int R);
// p = sc z32 + b p; umax (optional, zeroed by launch_dot2_zf_partial): max |p|
// per right-hand side for the next fixed-point stencil on p
void launch_axpby_zf(cudaStream_t s, int sm, int64_t N, const double* sc, const float* z32, const double* ab, double* p,
                     int R, unsigned long long* umax = nullptr);
void launch_to_f32(cudaStream_t s, int sm, int64_t N, const double* sc, const double* src, float* dst, int R);
void launch_from_f32(cudaStream_t s, int sm, int64_t N, const double* sc, const float* src, double* dst, int R);
void launch_add_f32(cudaStream_t s, int sm, int64_t N, const double* sc, const float* src, double* dst, int R);

}  // namespace ndmg
