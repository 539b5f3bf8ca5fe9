// C ABI of libndmg (include/ndmg.h): handle, level hierarchy, V-cycle driver
// (Fig. 1), PCG and the FP64 iterative-refinement loop.  All vector work runs
// in the kernels of kernels.cu / tc_patch.cu on the handle's stream.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <new>
#include <type_traits>

#include "coarse_cycle.cuh"
#include "kernels.cuh"
#include "tc_cell.cuh"
#include "tc_patch.cuh"

using namespace ndmg;

namespace {

int fail(ndmg_t* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(ndmg_t* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? NDMG_OUT_OF_MEMORY : NDMG_CUDA_ERROR, m);
}

#define NDMG_CK(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

// launch errors are sticky per call: check after queuing a group of launches
#define NDMG_CK_LAUNCH() NDMG_CK(cudaGetLastError())

// Counts launches and, when the class is traced, brackets them with events
// recorded on the handle's stream.
struct Span {
  ndmg_t* h;
  cudaEvent_t end = nullptr;
  bool external = false;  // recorded into a graph being captured
  Span(ndmg_t* h_, int cls, double units, int nlaunch = 1) : h(h_) {
    h->launch_total += nlaunch;
    if (!h->trace_on[cls]) return;
    if (h->capturing) {  // event-record nodes of the graph being captured
      ndmg_t::GraphSpan gs{cls, units, nlaunch, nullptr, nullptr};
      if (cudaEventCreate(&gs.a) != cudaSuccess) return;
      if (cudaEventCreate(&gs.b) != cudaSuccess) {
        cudaEventDestroy(gs.a);
        return;
      }
      cudaEventRecordWithFlags(gs.a, h->stream, cudaEventRecordExternal);
      h->vgraph_spans.push_back(gs);
      end = gs.b;
      external = true;
      return;
    }
    std::pair<cudaEvent_t, cudaEvent_t> pr{nullptr, nullptr};
    if (!h->ev_free.empty()) {
      pr = h->ev_free.back();
      h->ev_free.pop_back();
    } else if (cudaEventCreate(&pr.first) != cudaSuccess || cudaEventCreate(&pr.second) != cudaSuccess) {
      return;
    }
    h->trace_launches[cls] += nlaunch;
    h->trace_units[cls] += units;
    cudaEventRecord(pr.first, h->stream);
    h->ev_used[cls].push_back(pr);
    end = pr.second;
  }
  ~Span() {
    if (end && external) cudaEventRecordWithFlags(end, h->stream, cudaEventRecordExternal);
    else if (end) cudaEventRecord(end, h->stream);
  }
};

int collect_graph(ndmg_t* h);
void drop_graph(ndmg_t* h);

// NDMG_POISON_WORKSPACES=1 at ndmg_create: workspaces start as all-one bytes
bool poison_workspaces() {
  const char* v = std::getenv("NDMG_POISON_WORKSPACES");
  return v && v[0] == '1';
}

template <typename T>
T* dev_alloc(int64_t count, cudaError_t* err, bool poison = false) {
  void* p = nullptr;
  if (count <= 0) count = 1;
  cudaError_t e = cudaMalloc(&p, sizeof(T) * count);
  if (e == cudaSuccess && poison) e = cudaMemset(p, 0xFF, sizeof(T) * count);
  if (e != cudaSuccess && *err == cudaSuccess) *err = e;
  return (T*)p;
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<double>& src) {
  std::vector<T> tmp(src.size());
  for (size_t i = 0; i < src.size(); ++i) tmp[i] = (T)src[i];
  if (!*dst) {
    cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * tmp.size());
    if (e != cudaSuccess) return e;
  }
  return cudaMemcpy(*dst, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice);
}

// FP64 dense local operators (nl x nl each, `count` of them back to back in
// src) in the layout k_patch_dense_df reads: per operator the FP64 entries,
// then the float parts hi = fl(d) and lo = fl(d - hi) of every entry, i.e.
// dense_stride<double>(nl) doubles per operator
cudaError_t upload_dense64(double** dst, const std::vector<double>& src, int nl) {
  const size_t m = (size_t)nl * nl, count = src.size() / m;
  std::vector<double> tmp(count * dense_stride<double>(nl));
  for (size_t o = 0; o < count; ++o) {
    double* blk = tmp.data() + o * dense_stride<double>(nl);
    float* hl = reinterpret_cast<float*>(blk + m);
    for (size_t q = 0; q < m; ++q) {
      const double d = src[o * m + q];
      const float hi = (float)d;
      blk[q] = d;
      hl[q] = hi;
      hl[m + q] = (float)(d - (double)hi);
    }
  }
  if (!*dst) {
    cudaError_t e = cudaMalloc((void**)dst, sizeof(double) * tmp.size());
    if (e != cudaSuccess) return e;
  }
  return cudaMemcpy(*dst, tmp.data(), sizeof(double) * tmp.size(), cudaMemcpyHostToDevice);
}

// an FP64 dense patch operator in the mirror-symmetry basis of its box
// (words = 0: the dense double-float kernel is used instead)
cudaError_t upload_sym(uint32_t** dst, int* words, const PatchFamily& fam, const std::vector<double>& D) {
  std::vector<uint32_t> blob;
  double dropped = 0.0;
  // the off-block part of D is its set-up rounding (it is zero for the exact
  // operator); more than that means the box lacks the symmetry
  if (!build_patch_sym(fam, D.data(), &blob, &dropped) || !(dropped < 1e-6)) {
    *words = 0;
    return cudaSuccess;
  }
  if (*dst && *words != (int)blob.size()) {
    cudaFree(*dst);
    *dst = nullptr;
  }
  *words = (int)blob.size();
  blob.resize((blob.size() + 3) & ~(size_t)3, 0u);  // padded to 16 bytes for whole-chunk copies
  if (!*dst) {
    cudaError_t e = cudaMalloc((void**)dst, sizeof(uint32_t) * blob.size());
    if (e != cudaSuccess) return e;
  }
  return cudaMemcpy(*dst, blob.data(), sizeof(uint32_t) * blob.size(), cudaMemcpyHostToDevice);
}

// fresh device copy of a host array (any previous buffer freed first)
template <typename D, typename S>
cudaError_t upload_fresh(D** dst, const std::vector<S>& src) {
  cudaFree(*dst);
  *dst = nullptr;
  std::vector<D> tmp(src.begin(), src.end());
  if (tmp.empty()) tmp.resize(1);
  cudaError_t e = cudaMalloc((void**)dst, sizeof(D) * tmp.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, tmp.data(), sizeof(D) * tmp.size(), cudaMemcpyHostToDevice);
}

int64_t edges(int n) { return 3LL * n * (n - 1) * (n - 1); }
double bubble_bytes(int n, size_t w) {
  const double c = n / 2;
  return c * c * c * 18.0 * w;  // per coarse element: read 6 r, read+write 6 z
}
double num_patches(int n) {
  const double v = n / 2 - 1;
  return v > 0 ? v * v * v : 0.0;
}

// per-level FP64 / FP32 workspace pointers
template <typename T> T* lv_g(DevLevel& L);
template <typename T> T* lv_z(DevLevel& L);
template <typename T> T* lv_r(DevLevel& L);
template <> double* lv_g<double>(DevLevel& L) { return L.g64; }
template <> double* lv_z<double>(DevLevel& L) { return L.z64; }
template <> double* lv_r<double>(DevLevel& L) { return L.r64; }
template <> float* lv_g<float>(DevLevel& L) { return L.g32; }
template <> float* lv_z<float>(DevLevel& L) { return L.z32; }
template <> float* lv_r<float>(DevLevel& L) { return L.r32; }
const double* lv_Ainv(DevLevel& L, double*) { return L.AinvT64; }
const float* lv_Ainv(DevLevel& L, float*) { return L.AinvT32; }
const double* lv_D(DevLevel& L, double*) { return L.Dv64; }
const double* lv_De(DevLevel& L, double*) { return L.De64; }

bool mixed(const ndmg_t* h) {
  return h->o.precision == NDMG_PREC_MIXED_BF16 || h->o.precision == NDMG_PREC_MIXED_FP16;
}

// kernels with bounded device-side waits may have written the status word:
// the tensor-core smoothers (MIXED handles)
bool waits_on_device(const ndmg_t* h) { return mixed(h); }

// ---------------------------------------------------------------------------
// Level operations (every launch covers the R = nrhs right-hand sides)
// ---------------------------------------------------------------------------
int nrhs(const ndmg_t* h) { return h->o.nrhs; }

const double* lv_a(DevLevel& L, double*) { return L.a64; }
const float* lv_a(DevLevel& L, float*) { return L.a32; }

// y = g - (cK K + cM M) u (or (cK K + cM M) u when g is null) on level k: the
// constant-coefficient stencil, or with a coefficient per hexahedron the
// field stencil (cK = h times the factor; the coefficients are in K)
// (umax_ready: h->umax already holds max |u| per right-hand side)
template <typename T>
void stencil(ndmg_t* h, int k, double cK, double cM, const T* u, const T* g, T* y, bool umax_ready = false) {
  DevLevel& L = h->lv[k];
  const int kz = L.kz[sizeof(T) == 8 ? 1 : 0];
  if (h->field)
    launch_stencil_field<T>(h->stream, h->sm_count, L.n, cK, cM, u, g, y, nrhs(h), lv_a(L, (T*)nullptr), kz);
  else
    launch_stencil<T>(h->stream, h->sm_count, L.n, cK, cM, u, g, y, nrhs(h), h->umax, kz, umax_ready);
}

template <typename T>
void op_residual(ndmg_t* h, int k, const T* g, const T* z, T* r) {
  DevLevel& L = h->lv[k];
  Span sp(h, NDMG_K_STENCIL, 3.0 * sizeof(T) * L.N * nrhs(h));  // read g, z; write r
  stencil<T>(h, k, L.cK, L.cM, z, g, r);
}

template <typename T>
void op_apply(ndmg_t* h, int k, const T* x, T* y, bool umax_ready = false) {
  DevLevel& L = h->lv[k];
  Span sp(h, NDMG_K_STENCIL, 2.0 * sizeof(T) * L.N * nrhs(h));  // read x; write y
  stencil<T>(h, k, L.cK, L.cM, x, (const T*)nullptr, y, umax_ready);
}

// q = A p on the finest level for PCG, with the block partial sums of the
// curvature p.q formed in the same launch (fixed-point stencil) and left in
// h->pq_red; returns their number per right-hand side, 0 when the launch
// formed none (coefficient field, or more blocks than the buffer holds)
int op_apply_curvature(ndmg_t* h, const double* p, double* q, bool umax_ready) {
  const int K = h->K;
  DevLevel& L = h->lv[K];
  Span sp(h, NDMG_K_STENCIL, 2.0 * sizeof(double) * L.N * nrhs(h));  // read p; write q
  if (h->field) {
    stencil<double>(h, K, L.cK, L.cM, p, (const double*)nullptr, q, umax_ready);
    return 0;
  }
  return launch_stencil<double>(h->stream, h->sm_count, L.n, L.cK, L.cM, p, (const double*)nullptr, q, nrhs(h),
                                h->umax, L.kz[1], umax_ready, h->pq_red, h->pq_cap);
}

// alpha = rz / p.q on the device from the stencil's partial sums (nbq > 0)
// or from a separate reduction over p and q
void cg_alpha_device(ndmg_t* h, int nbq, const double* p, const double* q, const CgScalars& C, bool flex) {
  const int R = nrhs(h);
  const int64_t N = h->lv[h->K].N;
  if (nbq > 0) {
    Span sp(h, NDMG_K_BLAS, 0.0);
    launch_cg_scalars(h->stream, CG_ALPHA, nbq, h->pq_red, C, flex, h->status, R);
    return;
  }
  Span sp(h, NDMG_K_BLAS, 2.0 * 8 * N * R, 2);
  launch_dot2_partial<double>(h->stream, h->sm_count, N, p, q, nullptr, nullptr, h->red, R);
  launch_cg_scalars(h->stream, CG_ALPHA, reduction_blocks(h->sm_count), h->red, C, flex, h->status, R);
}

// y = g + (a K + b M) x (or (a K + b M) x when g is null): the stencil in
// residual form with the pencil's coefficients negated
template <typename T>
void op_pencil(ndmg_t* h, int k, double a, double b, const T* g, const T* x, T* y) {
  DevLevel& L = h->lv[k];
  const double hk = L.h, h3 = hk * hk * hk;
  Span sp(h, NDMG_K_STENCIL, (g ? 3.0 : 2.0) * sizeof(T) * L.N * nrhs(h));
  if (g) stencil<T>(h, k, -a * hk, -b * h3, x, g, y);
  else stencil<T>(h, k, a * hk, b * h3, x, (const T*)nullptr, y);
}

bool edge_smoother(const ndmg_t* h) { return h->o.smoother == NDMG_SMOOTHER_EDGE; }

// sum_E J_E A_E^{-1} J_E^t r of eq. (Preconditioner E): one launch per
// coarse-edge direction, each with its 42x42 operator
template <typename T>
void op_edge_terms(ndmg_t* h, int k, const T* De, const T* r, T* z) {
  DevLevel& L = h->lv[k];
  const int R = nrhs(h);
  for (int d = 0; d < 3; ++d) {
    const PatchFamily fam = edge_family(L.n, d);
    Span sp(h, NDMG_K_PATCH, (double)fam.np[0] * fam.np[1] * fam.np[2] * 2.0 * 42 * 42 * R);
    if constexpr (std::is_same<T, double>::value)
      if (L.sym_e_words[d] > 0) {
        launch_patch_sym(h->stream, h->sm_count, L.n, fam, L.sym_e[d], L.sym_e_words[d], h->o.eta, r, z, R);
        continue;
      }
    launch_patch_dense<T>(h->stream, h->sm_count, L.n, fam, De + d * dense_stride<T>(42), h->o.eta, r, z, R);
  }
}

// z += M_k^{-1} r (eta included), eq. (Preconditioner P) or (Preconditioner E)
// subdomain size 4 (CUDA cores in every precision mode): interior spaces of
// the 4x4x4 subdomains (108x108 dense) and the 1176-edge vertex patches in
// Gram form
const double* lv_Wg(DevLevel& L, double*) { return L.Wg64; }
const float* lv_Wg(DevLevel& L, float*) { return L.Wg32; }
const double* lv_WgT(DevLevel& L, double*) { return L.WgT64; }
const float* lv_WgT(DevLevel& L, float*) { return L.WgT32; }

template <typename T>
void op_smoother_s4(ndmg_t* h, int k, const T* r, T* z) {
  DevLevel& L = h->lv[k];
  const int R = nrhs(h);
  {
    const PatchFamily fam = subdomain4_family(L.n);
    Span sp(h, NDMG_K_BUBBLE, (double)fam.np[0] * fam.np[1] * fam.np[2] * 2.0 * 108 * 108 * R);
    bool done = false;
    if constexpr (std::is_same<T, double>::value)
      if (L.sym_s4_words > 0) {
        launch_patch_sym(h->stream, h->sm_count, L.n, fam, L.sym_s4, L.sym_s4_words, h->o.eta, r, z, R);
        done = true;
      }
    if (!done) launch_patch_dense<T>(h->stream, h->sm_count, L.n, fam, lv_Ainv(L, (T*)nullptr), h->o.eta, r, z, R);
  }
  const PatchFamily fam = vertex4_family(L.n);
  Span sp(h, NDMG_K_PATCH, (double)fam.np[0] * fam.np[1] * fam.np[2] * 4.0 * 1176 * 312 * R);
  launch_patch_gram<T>(h->stream, h->sm_count, L.n, fam, 312, lv_Wg(L, (T*)nullptr), lv_WgT(L, (T*)nullptr),
                       h->o.eta, r, z, R);
}

// coefficient per hexahedron: interior solves and patch solves with one
// operator per group of subdomains / patches (tensor cores for the vertex
// patches in the MIXED modes)
const double* lv_bubA(DevLevel& L, double*) { return L.bubA64; }
const float* lv_bubA(DevLevel& L, float*) { return L.bubA32; }
const double* grp_op(DevGrouped& G, double*) { return G.op64; }
const float* grp_op(DevGrouped& G, float*) { return G.op32; }

template <typename T>
void op_smoother_field(ndmg_t* h, int k, const T* r, T* z) {
  DevLevel& L = h->lv[k];
  const int R = nrhs(h);
  if constexpr (std::is_same<T, float>::value) {
    if (mixed(h) && !edge_smoother(h) && L.Wtc_tab && L.tc) {
      Span sp(h, NDMG_K_PATCH, 12.0 * L.N * R);
      launch_tc_smoother_field(h->stream, L.n, L.Wtc_tab, h->o.precision == NDMG_PREC_MIXED_FP16, L.bubA32,
                               L.bub_gid, L.tc_off, L.tc_grp, L.tc_mask, h->o.eta, r, z, h->status, R);
      return;
    }
  }
  {
    Span sp(h, NDMG_K_BUBBLE, bubble_bytes(L.n, sizeof(T)) * R);
    launch_bubble_grouped<T>(h->stream, h->sm_count, L.n, lv_bubA(L, (T*)nullptr), L.bub_gid, h->o.eta, r, z, R);
  }
  if (edge_smoother(h)) {
    for (int d = 0; d < 3; ++d) {
      const PatchFamily fam = edge_family(L.n, d);
      Span sp(h, NDMG_K_PATCH, (double)fam.np[0] * fam.np[1] * fam.np[2] * 2.0 * 42 * 42 * R);
      launch_patch_grouped<T>(h->stream, h->sm_count, L.n, fam, grp_op(L.edg[d], (T*)nullptr), L.edg[d].chunks,
                              L.edg[d].nchunks, L.edg[d].plist, h->o.eta, r, z, R);
    }
    return;
  }
  const PatchFamily fam = vertex_family(L.n);
  Span sp(h, NDMG_K_PATCH, mixed(h) && sizeof(T) == 4 ? 12.0 * L.N * R : num_patches(L.n) * 2.0 * 108 * 108 * R);
  launch_patch_grouped<T>(h->stream, h->sm_count, L.n, fam, grp_op(L.vtx, (T*)nullptr), L.vtx.chunks, L.vtx.nchunks,
                          L.vtx.plist, h->o.eta, r, z, R);
}

template <typename T>
void op_smoother(ndmg_t* h, int k, const T* r, T* z) {
  DevLevel& L = h->lv[k];
  const int R = nrhs(h);
  if (h->field) {
    op_smoother_field<T>(h, k, r, z);
    return;
  }
  if (h->o.subdomain == 4) {
    op_smoother_s4<T>(h, k, r, z);
    return;
  }
  if constexpr (std::is_same<T, double>::value)
    if (L.sym_v_words > 0 && !edge_smoother(h)) {
      // the vertex patches in the mirror-symmetry basis and the interior
      // solves of the coarse elements in one launch
      Span sp(h, NDMG_K_PATCH, num_patches(L.n) * 2.0 * 108 * 108 * R);  // dense-equivalent 108x108 per patch
      launch_patch_sym(h->stream, h->sm_count, L.n, vertex_family(L.n), L.sym_v, L.sym_v_words, h->o.eta, r, z, R,
                       L.AinvT64);
      return;
    }
  {
    Span sp(h, NDMG_K_BUBBLE, bubble_bytes(L.n, sizeof(T)) * R);
    launch_bubble<T>(h->stream, h->sm_count, L.n, lv_Ainv(L, (T*)nullptr), h->o.eta, r, z, R);
  }
  if (edge_smoother(h)) {
    op_edge_terms<T>(h, k, lv_De(L, (T*)nullptr), r, z);
    return;
  }
  Span sp(h, NDMG_K_PATCH, num_patches(L.n) * 2.0 * 108 * 108 * R);  // dense 108x108 per patch
  launch_vertex_dense<T>(h->stream, h->sm_count, L.n, lv_D(L, (T*)nullptr), h->o.eta, r, z, R);
}

template <>
void op_smoother<float>(ndmg_t* h, int k, const float* r, float* z) {
  DevLevel& L = h->lv[k];
  const int R = nrhs(h);
  if (h->field) {
    op_smoother_field<float>(h, k, r, z);
    return;
  }
  if (h->o.subdomain == 4) {
    op_smoother_s4<float>(h, k, r, z);
    return;
  }
  if (edge_smoother(h)) {  // the edge-based smoother runs on CUDA cores in every precision mode
    {
      Span sp(h, NDMG_K_BUBBLE, bubble_bytes(L.n, sizeof(float)) * R);
      launch_bubble<float>(h->stream, h->sm_count, L.n, L.AinvT32, h->o.eta, r, z, R);
    }
    op_edge_terms<float>(h, k, L.De32, r, z);
    return;
  }
  if (mixed(h) && L.tc && L.tc_kind == 2 && L.Wcell) {
    // vertex patches on tensor cores (Gram form W W^t, cell-owned rows:
    // shifted-row GEMMs, one writer per edge) and the interior 6x6 solves in
    // one persistent kernel.  Algorithmic bytes: read r, read and write z
    // (FP32); 25,920 flops per patch is ~86 flop/B, below the bf16 ridge of
    // ~256 flop/B, so the work is memory-bound.
    Span sp(h, NDMG_K_PATCH, 12.0 * L.N * R);
    launch_tc_cell_smoother(h->stream, h->sm_count, L.n, L.Wcell, h->o.precision == NDMG_PREC_MIXED_FP16, L.AinvT32,
                            h->o.eta, r, z, h->status, R, L.zlen);
    return;
  }
  if (mixed(h) && L.tc && L.Wtc) {
    // the same on tensor cores per brick of 128 vertex patches (gathered
    // operand, shared-memory accumulation, global reductions)
    Span sp(h, NDMG_K_PATCH, 12.0 * L.N * R);
    launch_tc_smoother(h->stream, h->sm_count, L.n, L.Wtc, h->o.precision == NDMG_PREC_MIXED_FP16, L.AinvT32,
                       h->o.eta, r, z, h->status, R);
    return;
  }
  if (L.sym_v_words > 0) {
    // interior and patch solves in one launch, the patch operator in the
    // basis of the patch's mirror symmetries (FP32 block products)
    Span sp(h, NDMG_K_PATCH, mixed(h) ? 12.0 * L.N * R : num_patches(L.n) * 2.0 * 108 * 108 * R);
    launch_smooth_sym32(h->stream, L.n, L.sym_v, L.sym_v_words, L.AinvT32, h->o.eta, r, z, R);
    return;
  }
  if (smooth_direct_fits(L.n)) {
    // a small level: interior and patch solves in one launch, the operator
    // staged in shared memory
    Span sp(h, NDMG_K_PATCH, mixed(h) ? 12.0 * L.N * R : num_patches(L.n) * 2.0 * 108 * 108 * R);
    launch_smooth_direct(h->stream, L.n, L.Dv32, L.AinvT32, h->o.eta, r, z, R);
    return;
  }
  {
    Span sp(h, NDMG_K_BUBBLE, bubble_bytes(L.n, sizeof(float)) * R);
    launch_bubble<float>(h->stream, h->sm_count, L.n, L.AinvT32, h->o.eta, r, z, R);
  }
  // MIXED handles (a level where the autotuner preferred these kernels) count
  // the smoother's algorithmic bytes here, as for the tensor-core kernel;
  // FP32 handles count flops
  Span sp(h, NDMG_K_PATCH, mixed(h) ? 12.0 * L.N * R : num_patches(L.n) * 2.0 * 108 * 108 * R);
  launch_vertex_dense<float>(h->stream, h->sm_count, L.n, L.Dv32, h->o.eta, r, z, R);
}

template <typename T>
void op_smooth_steps(ndmg_t* h, int k, const T* g, T* z, int steps) {
  T* r = lv_r<T>(h->lv[k]);
  for (int s = 0; s < steps; ++s) {
    op_residual<T>(h, k, g, z, r);
    op_smoother<T>(h, k, r, z);
  }
}

// the small-level cluster kernel serves float V-cycles on levels 1 .. Kc
// that start from z = 0 (constant coefficient, vertex smoother, subdomain 2)
bool coarse_cycle_on(const ndmg_t* h, int k) {
  return h->coarse_on && h->Kc > 0 && k >= 1 && k <= h->Kc && h->coarse_grid > 0 && !h->field;
}

// z = MG(k, g, 0, m) for k <= Kc in one cluster launch
void op_coarse_cycle(ndmg_t* h, int k, const float* g, float* z) {
  CoarseLevel cl[kCoarseMaxLevels + 1];
  double units = 0.0;
  for (int j = 0; j <= k; ++j) {
    DevLevel& L = h->lv[j];
    cl[j].n = L.n;
    cl[j].cK = L.cK;
    cl[j].cM = L.cM;
    cl[j].g = j == k ? const_cast<float*>(g) : L.g32;
    cl[j].z = j == k ? z : L.z32;
    cl[j].r = L.r32;
    cl[j].W = L.Wv32;
    cl[j].AinvT = L.AinvT32;
    units += 74.0 * L.N * nrhs(h);   // FP32 bytes of one V-cycle level (read / write of g, z, r)
  }
  Span sp(h, NDMG_K_COARSE, units);
  launch_coarse_cycle(h->stream, h->coarse_grid, cl, k, (int)h->lv[0].N, h->Ainv0, h->lv[0].g32, h->lv[0].z32,
                      h->o.eta, h->o.m, nrhs(h), h->status);
}

// MG(k, g, z, m) of Fig. 1 with z in/out; z_zero: z is 0 on entry, so the
// first pre-smoothing residual is g itself (no stencil pass)
template <typename T>
void op_vcycle(ndmg_t* h, int k, const T* g, T* z, bool z_zero = false) {
  const int R = nrhs(h);
  if (k == h->K) ++h->vcycle_total;
  if constexpr (std::is_same<T, float>::value) {
    if (z_zero && coarse_cycle_on(h, k)) {
      op_coarse_cycle(h, k, g, z);
      return;
    }
  }
  if (k == 0) {
    const double N0 = (double)h->lv[0].N;
    Span sp(h, NDMG_K_COARSE, (2.0 * sizeof(T) * N0 + 8.0 * N0 * N0) * R);
    launch_coarse<T>(h->stream, (int)h->lv[0].N, h->Ainv0, g, z, R);
    return;
  }
  DevLevel& L = h->lv[k];
  DevLevel& C = h->lv[k - 1];
  T* r = lv_r<T>(L);
  if (z_zero) {
    op_smoother<T>(h, k, g, z);
    op_smooth_steps<T>(h, k, g, z, h->o.m - 1);
  } else {
    op_smooth_steps<T>(h, k, g, z, h->o.m);
  }
  op_residual<T>(h, k, g, z, r);
  {
    // the restriction also zeroes the coarse solution (no memset between
    // dependent launches)
    Span sp(h, NDMG_K_RESTRICT, (double)sizeof(T) * (L.N + 2 * C.N) * R);
    launch_restrict<T>(h->stream, h->sm_count, L.n, r, lv_g<T>(C), R, lv_z<T>(C));
  }
  op_vcycle<T>(h, k - 1, lv_g<T>(C), lv_z<T>(C), true);
  {
    Span sp(h, NDMG_K_PROLONG, (double)sizeof(T) * (2 * L.N + C.N) * R);
    launch_prolong_add<T>(h->stream, h->sm_count, L.n, lv_z<T>(C), z, R);
  }
  op_smooth_steps<T>(h, k, g, z, h->o.m);
}

// per-right-hand-side FP64 inner products x_r.y_r (and x2_r.y2_r), synchronised
template <typename T>
int dot2(ndmg_t* h, int64_t N, const T* x, const T* y, const T* x2, const T* y2, std::vector<double>& a,
         std::vector<double>* b) {
  const int R = nrhs(h);
  const int nb = reduction_blocks(h->sm_count);
  double* out = h->red + 2 * (int64_t)nb * R;
  {
    Span sp(h, NDMG_K_BLAS, (double)sizeof(T) * N * (x2 ? 4 : 2) * R, 2);
    launch_dot2<T>(h->stream, h->sm_count, N, x, y, x2, y2, h->red, out, R);
  }
  NDMG_CK_LAUNCH();
  NDMG_CK(cudaMemcpyAsync(h->red_host, out, 2 * sizeof(double) * R, cudaMemcpyDeviceToHost, h->stream));
  NDMG_CK(cudaStreamSynchronize(h->stream));
  if (int st = collect_graph(h)) return st;
  a.resize(R);
  if (b) b->resize(R);
  for (int i = 0; i < R; ++i) {
    a[i] = h->red_host[2 * i];
    if (b) (*b)[i] = h->red_host[2 * i + 1];
  }
  return NDMG_OK;
}

// reads the per-right-hand-side sums a kernel pair left in out[2 r], [2 r + 1]
// (and, with status, the device status word in the same synchronisation)
int read_sums(ndmg_t* h, const double* out, std::vector<double>& a, std::vector<double>* b, bool status) {
  const int R = nrhs(h);
  NDMG_CK_LAUNCH();
  NDMG_CK(cudaMemcpyAsync(h->red_host, out, 2 * sizeof(double) * R, cudaMemcpyDeviceToHost, h->stream));
  if (status) NDMG_CK(cudaMemcpyAsync(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  NDMG_CK(cudaStreamSynchronize(h->stream));
  if (int st = collect_graph(h)) return st;
  if (status && *h->status_host != 0) {
    const int code = *h->status_host;
    cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
    return fail(h, NDMG_DEVICE_TIMEOUT, "a device-side wait timed out (status " + std::to_string(code) + ")");
  }
  a.resize(R);
  if (b) b->resize(R);
  for (int i = 0; i < R; ++i) {
    a[i] = h->red_host[2 * i];
    if (b) (*b)[i] = h->red_host[2 * i + 1];
  }
  return NDMG_OK;
}

// per-right-hand-side scalars for the BLAS kernels: each purpose has its own
// pinned and device slot, rewritten only after a synchronisation that
// follows its previous use
enum CoefSlot { SLOT_ALPHA = 0, SLOT_AB = 1, SLOT_TO = 2, SLOT_FROM = 3, SLOT_COUNT = 4 };

const double* push_coef(ndmg_t* h, int slot, const std::vector<double>& v) {
  const int R = nrhs(h);
  double* hp = h->coef_host + (size_t)slot * 2 * R;
  double* dp = h->coef + (size_t)slot * 2 * R;
  std::memcpy(hp, v.data(), sizeof(double) * v.size());
  cudaMemcpyAsync(dp, hp, sizeof(double) * v.size(), cudaMemcpyHostToDevice, h->stream);
  return dp;
}

// device PCG scalars of the handle
CgScalars cg_scalars(ndmg_t* h) {
  const int R = nrhs(h);
  double* b = h->cg;
  return CgScalars{b, b + R, b + 3 * R, b + 4 * R, b + 5 * R, b + 6 * R, b + 7 * R};
}

// writes rr, rz and the done flags of every right-hand side to the device
int cg_push_state(ndmg_t* h, const std::vector<double>& rr, const std::vector<double>& rz,
                  const std::vector<char>& done) {
  const int R = nrhs(h);
  const CgScalars S = cg_scalars(h);
  double* hp = h->cg_host;
  for (int i = 0; i < R; ++i) {
    hp[i] = rr[i];
    hp[R + i] = rz[i];
    hp[2 * R + i] = done[i] ? 1.0 : 0.0;
  }
  NDMG_CK(cudaMemcpyAsync(S.rr, hp, sizeof(double) * R, cudaMemcpyHostToDevice, h->stream));
  NDMG_CK(cudaMemcpyAsync(S.rz, hp + R, sizeof(double) * R, cudaMemcpyHostToDevice, h->stream));
  NDMG_CK(cudaMemcpyAsync(S.done, hp + 2 * R, sizeof(double) * R, cudaMemcpyHostToDevice, h->stream));
  NDMG_CK(cudaStreamSynchronize(h->stream));   // the pinned buffer is reused right away
  return NDMG_OK;
}

// the one synchronisation of a PCG iteration: rr of every right-hand side and
// the status word (a breakdown the device detected, a device-side timeout)
int cg_read_rr(ndmg_t* h, std::vector<double>& rr) {
  const int R = nrhs(h);
  const CgScalars S = cg_scalars(h);
  NDMG_CK_LAUNCH();
  NDMG_CK(cudaMemcpyAsync(h->cg_host, S.rr, sizeof(double) * R, cudaMemcpyDeviceToHost, h->stream));
  NDMG_CK(cudaMemcpyAsync(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  NDMG_CK(cudaStreamSynchronize(h->stream));
  if (int st = collect_graph(h)) return st;
  if (const int code = *h->status_host) {
    cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
    if (code & kStatusBreakdown) return fail(h, NDMG_BREAKDOWN, "non-positive curvature p^T A p");
    return fail(h, NDMG_DEVICE_TIMEOUT, "a device-side wait timed out (status " + std::to_string(code) + ")");
  }
  rr.assign(h->cg_host, h->cg_host + R);
  return NDMG_OK;
}

// done flags to the device after a convergence check (pinned staging slot
// 2R.., rewritten only after the next synchronisation)
int cg_push_done(ndmg_t* h, const std::vector<char>& done) {
  const int R = nrhs(h);
  double* hp = h->cg_host + 2 * R;
  for (int i = 0; i < R; ++i) hp[i] = done[i] ? 1.0 : 0.0;
  NDMG_CK(cudaMemcpyAsync(cg_scalars(h).done, hp, sizeof(double) * R, cudaMemcpyHostToDevice, h->stream));
  return NDMG_OK;
}

int check_level(ndmg_t* h, int32_t& level, bool need_fine_transfer) {
  if (level == -1) level = h->K;
  if (level < 0 || level > h->K) return fail(h, NDMG_INVALID_ARG, "level out of range");
  if (need_fine_transfer && level < 1) return fail(h, NDMG_INVALID_ARG, "level must be >= 1");
  return NDMG_OK;
}

int check_dtype(ndmg_t* h, int32_t dtype) {
  if (dtype != NDMG_F64 && dtype != NDMG_F32) return fail(h, NDMG_INVALID_ARG, "dtype must be NDMG_F64 or NDMG_F32");
  return NDMG_OK;
}

bool misaligned(const void* p) { return p == nullptr || ((uintptr_t)p & 15u) != 0; }

int check_ptrs(ndmg_t* h, std::initializer_list<const void*> ps) {
  for (const void* p : ps)
    if (misaligned(p)) return fail(h, NDMG_INVALID_ARG, "vector pointer is NULL or not 16-byte aligned");
  return NDMG_OK;
}

int check_status(ndmg_t* h) {
  NDMG_CK(cudaMemcpyAsync(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  NDMG_CK(cudaStreamSynchronize(h->stream));
  const int st = *h->status_host;
  if (st != 0) {
    cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
    return fail(h, NDMG_DEVICE_TIMEOUT, "a device-side wait timed out (status " + std::to_string(st) + ")");
  }
  return NDMG_OK;
}

double max_of(const std::vector<double>& v) {
  double m = 0.0;
  for (double x : v) m = std::isfinite(x) ? std::fmax(m, x) : x;
  return m;
}

// ---------------------------------------------------------------------------
// Solvers.  All right-hand sides iterate in lockstep, each with its own
// scalars; a right-hand side that has converged is frozen (alpha = beta = 0)
// while the others continue.
// ---------------------------------------------------------------------------
struct CGState {
  std::vector<double> nf, rz, relres;
  std::vector<char> done;
};

// one CG scalar update for every right-hand side; returns BREAKDOWN on a
// non-positive or non-finite curvature of a live right-hand side
int cg_alpha(ndmg_t* h, CGState& S, const std::vector<double>& pq, std::vector<double>& a) {
  const int R = nrhs(h);
  a.assign(R, 0.0);
  for (int i = 0; i < R; ++i) {
    if (S.done[i]) continue;
    if (!(pq[i] > 0.0) || !std::isfinite(pq[i])) return fail(h, NDMG_BREAKDOWN, "non-positive curvature p^T A p");
    a[i] = S.rz[i] / pq[i];
  }
  return NDMG_OK;
}

// relative residuals from ||r||^2; marks converged right-hand sides
int cg_check(ndmg_t* h, CGState& S, const std::vector<double>& rr, double tol, bool* all_done) {
  const int R = nrhs(h);
  *all_done = true;
  for (int i = 0; i < R; ++i) {
    S.relres[i] = std::sqrt(rr[i]) / S.nf[i];
    if (!std::isfinite(S.relres[i])) return fail(h, NDMG_BREAKDOWN, "non-finite residual");
    if (S.relres[i] <= tol) S.done[i] = 1;
    *all_done = *all_done && S.done[i];
  }
  return NDMG_OK;
}

int cg_init(ndmg_t* h, CGState& S, const std::vector<double>& ff, const std::vector<double>& rr, double tol,
            bool* all_done) {
  const int R = nrhs(h);
  S.nf.resize(R);
  S.rz.assign(R, 0.0);
  S.relres.assign(R, 0.0);
  S.done.assign(R, 0);
  for (int i = 0; i < R; ++i) S.nf[i] = std::sqrt(ff[i]) > 0 ? std::sqrt(ff[i]) : 1.0;
  return cg_check(h, S, rr, tol, all_done);
}

// FP64 PCG preconditioned by one FP64 V-cycle.  The scalars alpha, beta
// and rz live on the device (k_cg_scalars); each iteration reads back only
// ||r||^2 (and the status word) for the convergence test.
int pcg64(ndmg_t* h, const double* f, double* u, double tol, int maxit, int* iters, double* relres) {
  const int K = h->K, R = nrhs(h);
  const int64_t N = h->lv[K].N;
  const int sm = h->sm_count, nb = reduction_blocks(sm);
  double *r = h->w64[0], *z = h->w64[1], *p = h->w64[2], *q = h->w64[3];
  std::vector<double> ff, rr, rz0;
  CGState S;
  bool all_done = false;
  int st;
  *iters = 0;
  op_residual<double>(h, K, f, u, r);
  if ((st = dot2<double>(h, N, f, f, r, r, ff, &rr)) != NDMG_OK) return st;
  if ((st = cg_init(h, S, ff, rr, tol, &all_done)) != NDMG_OK) return st;
  *relres = max_of(S.relres);
  if (all_done) return NDMG_OK;
  cudaMemsetAsync(z, 0, sizeof(double) * N * R, h->stream);
  op_vcycle<double>(h, K, r, z, true);
  if ((st = dot2<double>(h, N, r, z, (const double*)nullptr, (const double*)nullptr, rz0, nullptr)) != NDMG_OK)
    return st;
  if ((st = cg_push_state(h, rr, rz0, S.done)) != NDMG_OK) return st;
  NDMG_CK(cudaMemcpyAsync(p, z, sizeof(double) * N * R, cudaMemcpyDeviceToDevice, h->stream));
  const CgScalars C = cg_scalars(h);
  // from the second iteration on, the update that forms p also forms the
  // fixed-point stencil's max |p| (no separate pass over p); the coefficient
  // field's FP64 stencil runs in plain FP64 and needs none
  const bool fuse_max = !h->field;
  for (int it = 1; it <= maxit; ++it) {
    const int nbq = op_apply_curvature(h, p, q, fuse_max && it > 1);
    cg_alpha_device(h, nbq, p, q, C, false);
    {
      Span sp(h, NDMG_K_BLAS, 6.0 * 8 * N * R);
      launch_cg_update<double>(h->stream, sm, N, C.alpha, p, q, u, r, R);
    }
    {
      Span sp(h, NDMG_K_BLAS, 1.0 * 8 * N * R, 2);
      launch_dot2_partial<double>(h->stream, sm, N, r, r, nullptr, nullptr, h->red, R);
      launch_cg_scalars(h->stream, CG_RR, nb, h->red, C, false, h->status, R);
    }
    if ((st = cg_read_rr(h, rr)) != NDMG_OK) return st;
    *iters = it;
    if ((st = cg_check(h, S, rr, tol, &all_done)) != NDMG_OK) return st;
    *relres = max_of(S.relres);
    if (all_done) return NDMG_OK;
    if ((st = cg_push_done(h, S.done)) != NDMG_OK) return st;
    cudaMemsetAsync(z, 0, sizeof(double) * N * R, h->stream);
    op_vcycle<double>(h, K, r, z, true);
    {
      Span sp(h, NDMG_K_BLAS, 2.0 * 8 * N * R, 2);
      launch_dot2_partial<double>(h->stream, sm, N, r, z, nullptr, nullptr, h->red, R);
      launch_cg_scalars(h->stream, CG_BETA, nb, h->red, C, false, h->status, R);
    }
    {
      Span sp(h, NDMG_K_BLAS, 3.0 * 8 * N * R);
      launch_axpby<double>(h->stream, sm, N, C.ab, z, p, R);
    }
  }
  return fail(h, NDMG_NOT_CONVERGED, "PCG reached maxit");
}

// the float V-cycle as preconditioner of FP64 vectors: z = ||r|| MG(r / ||r||)
// CUDA graph of the float V-cycle on the finest level (r32 -> z32, z32 = 0
// on entry): built on first use, dropped when the operators or the tracing
// change
void drop_graph(ndmg_t* h) {
  if (h->vgraph) cudaGraphExecDestroy(h->vgraph);
  h->vgraph = nullptr;
  for (auto& gs : h->vgraph_spans) {
    cudaEventDestroy(gs.a);
    cudaEventDestroy(gs.b);
  }
  h->vgraph_spans.clear();
  h->graph_pending = false;
}

// adds the traced times of the last replay (call after a synchronisation)
int collect_graph(ndmg_t* h) {
  if (!h->graph_pending) return NDMG_OK;
  h->graph_pending = false;
  for (auto& gs : h->vgraph_spans) {
    float t = 0.f;
    NDMG_CK(cudaEventElapsedTime(&t, gs.a, gs.b));
    h->trace_ms_graph[gs.cls] += t;
    h->trace_launches[gs.cls] += gs.nlaunch;
    h->trace_units[gs.cls] += gs.units;
  }
  return NDMG_OK;
}

// z32 = MG(K, r32, 0, m) on the handle's float work vectors w32[4] -> w32[5]
int vcycle_f32_graph(ndmg_t* h) {
  const int K = h->K, R = nrhs(h);
  const int64_t N = h->lv[K].N;
  float *r32 = h->w32[4], *z32 = h->w32[5];
  if (!h->use_graphs) {
    cudaMemsetAsync(z32, 0, sizeof(float) * N * R, h->stream);
    op_vcycle<float>(h, K, r32, z32, true);
    return NDMG_OK;
  }
  if (h->graph_pending) {  // the previous replay's events are about to be reused
    NDMG_CK(cudaStreamSynchronize(h->stream));
    if (int st = collect_graph(h)) return st;
  }
  if (!h->vgraph) {
    // captured on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured), replayed on the caller's
    if (!h->cap_stream) NDMG_CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const int64_t l0 = h->launch_total, v0 = h->vcycle_total;
    cudaStream_t user = h->stream;
    NDMG_CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
    h->stream = h->cap_stream;
    h->capturing = true;
    cudaMemsetAsync(z32, 0, sizeof(float) * N * R, h->stream);
    op_vcycle<float>(h, K, r32, z32, true);
    h->capturing = false;
    h->stream = user;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->vgraph, g, 0);
    if (g) cudaGraphDestroy(g);
    h->vgraph_launches = h->launch_total - l0;
    h->vgraph_vcycles = h->vcycle_total - v0;
    h->launch_total = l0;
    h->vcycle_total = v0;
    if (e != cudaSuccess) {
      // this stream cannot capture the V-cycle's launches: replay them
      // directly from now on
      drop_graph(h);
      cudaGetLastError();
      h->use_graphs = false;
      cudaMemsetAsync(z32, 0, sizeof(float) * N * R, h->stream);
      op_vcycle<float>(h, K, r32, z32, true);
      return NDMG_OK;
    }
  }
  NDMG_CK(cudaGraphLaunch(h->vgraph, h->stream));
  h->launch_total += h->vgraph_launches;
  h->vcycle_total += h->vgraph_vcycles;
  h->graph_pending = !h->vgraph_spans.empty();
  return NDMG_OK;
}

int precondition_mixed(ndmg_t* h, const double* r, double* z, const std::vector<double>& rnorm) {
  const int K = h->K, R = nrhs(h);
  const int64_t N = h->lv[K].N;
  const int sm = h->sm_count;
  float *r32 = h->w32[4], *z32 = h->w32[5];
  // power-of-two scales 2^-e, 2^e with 2^(e-1) <= ||r|| < 2^e (as the
  // device forms them for the later iterations, k_cg_scalars)
  std::vector<double> inv(R), fwd(R);
  for (int i = 0; i < R; ++i) {
    if (rnorm[i] > 0 && std::isfinite(rnorm[i])) {
      const int e = std::min(1022, std::max(-1022, std::ilogb(rnorm[i]) + 1));
      inv[i] = std::ldexp(1.0, -e);
      fwd[i] = std::ldexp(1.0, e);
    } else {
      inv[i] = 0.0;
      fwd[i] = rnorm[i];
    }
  }
  {
    const double* d = push_coef(h, SLOT_TO, inv);
    Span sp(h, NDMG_K_BLAS, 12.0 * N * R);
    launch_to_f32(h->stream, sm, N, d, r, r32, R);
  }
  if (int st = vcycle_f32_graph(h)) return st;
  {
    const double* d = push_coef(h, SLOT_FROM, fwd);
    Span sp(h, NDMG_K_BLAS, 12.0 * N * R);
    launch_from_f32(h->stream, sm, N, d, z32, z, R);
  }
  return waits_on_device(h) ? check_status(h) : NDMG_OK;
}

// FP64 flexible PCG preconditioned by the float V-cycle (mixed handles):
// r, p, q, u and every inner product stay in double; the preconditioner sees
// 2^-e r in float with 2^(e-1) <= ||r|| < 2^e (keeps fp16 operands in range;
// a power of two, so both scalings are exact exponent shifts) and returns z
// in double.
// beta = -a (q . z_new) / (r . z)_old (flexible form: the low-precision
// V-cycle is symmetric only up to rounding).  The scalars live on the device
// (k_cg_scalars); each iteration reads back only ||r||^2 and the status word.
int pcg_mixed(ndmg_t* h, const double* f, double* u, double tol, int maxit, int* iters, double* relres) {
  const int K = h->K, R = nrhs(h);
  const int64_t N = h->lv[K].N;
  const int sm = h->sm_count, nb = reduction_blocks(sm);
  double *r = h->w64[0], *z = h->w64[1], *p = h->w64[2], *q = h->w64[3];
  std::vector<double> ff, rr, rz0, rn(R);
  CGState S;
  bool all_done = false;
  int st;
  *iters = 0;
  op_residual<double>(h, K, f, u, r);
  if ((st = dot2<double>(h, N, f, f, r, r, ff, &rr)) != NDMG_OK) return st;
  if ((st = cg_init(h, S, ff, rr, tol, &all_done)) != NDMG_OK) return st;
  *relres = max_of(S.relres);
  if (all_done) return NDMG_OK;
  for (int i = 0; i < R; ++i) rn[i] = std::sqrt(rr[i]);
  if ((st = precondition_mixed(h, r, z, rn)) != NDMG_OK) return st;
  if ((st = dot2<double>(h, N, r, z, (const double*)nullptr, (const double*)nullptr, rz0, nullptr)) != NDMG_OK)
    return st;
  if ((st = cg_push_state(h, rr, rz0, S.done)) != NDMG_OK) return st;
  NDMG_CK(cudaMemcpyAsync(p, z, sizeof(double) * N * R, cudaMemcpyDeviceToDevice, h->stream));
  // per iteration: q = A p; alpha = rz / (p.q) and the scales 1 / ||r||,
  // ||r|| of the current residual (device); u, r update fused with (r.r) and
  // the float right-hand side of the V-cycle; the one read-back; V-cycle;
  // (r.z), (q.z) and beta (device); p = z + beta p straight from the float
  // V-cycle output
  float* z32 = h->w32[5];
  const CgScalars C = cg_scalars(h);
  // from the second iteration on, the update that forms p also forms the
  // fixed-point stencil's max |p| (no separate pass over p); the coefficient
  // field's FP64 stencil runs in plain FP64 and needs none
  const bool fuse_max = !h->field;
  for (int it = 1; it <= maxit; ++it) {
    const int nbq = op_apply_curvature(h, p, q, fuse_max && it > 1);
    cg_alpha_device(h, nbq, p, q, C, true);
    {
      Span sp(h, NDMG_K_BLAS, (6.0 * 8 + 4) * N * R, 2);
      launch_cg_update_rr_partial(h->stream, sm, N, C.alpha, p, q, u, r, C.sto, h->w32[4], h->red, R);
      launch_cg_scalars(h->stream, CG_RR, nb, h->red, C, true, h->status, R);
    }
    if ((st = cg_read_rr(h, rr)) != NDMG_OK) return st;
    *iters = it;
    if ((st = cg_check(h, S, rr, tol, &all_done)) != NDMG_OK) return st;
    *relres = max_of(S.relres);
    if (all_done) return NDMG_OK;
    if ((st = cg_push_done(h, S.done)) != NDMG_OK) return st;
    // z = ||r_old|| z32 with z32 = V-cycle(r / ||r_old||)
    if ((st = vcycle_f32_graph(h)) != NDMG_OK) return st;
    {
      Span sp(h, NDMG_K_BLAS, (2.0 * 8 + 4) * N * R, 2);
      launch_dot2_zf_partial(h->stream, sm, N, r, q, z32, h->red, R, fuse_max ? h->umax : nullptr);
      launch_cg_scalars(h->stream, CG_BETA_FLEX, nb, h->red, C, true, h->status, R);
    }
    {
      Span sp(h, NDMG_K_BLAS, (2.0 * 8 + 4) * N * R);
      launch_axpby_zf(h->stream, sm, N, C.sfrom, z32, C.ab, p, R, fuse_max ? h->umax : nullptr);
    }
  }
  return fail(h, NDMG_NOT_CONVERGED, "PCG reached maxit");
}

// float PCG on A d = b (b float, d float, d starts at 0) to relative tol;
// flexible beta.  Returns OK also when maxit is reached: the outer
// refinement loop judges convergence.
int pcg32(ndmg_t* h, const float* b, float* d, double tol, int maxit, int* iters) {
  const int K = h->K, R = nrhs(h);
  const int64_t N = h->lv[K].N;
  const int sm = h->sm_count;
  float *r = h->w32[0], *z = h->w32[1], *p = h->w32[2], *q = h->w32[3];
  std::vector<double> bb, rr, pq, rz_new, qz, a, ab(2 * R);
  CGState S;
  bool all_done = false;
  int st;
  *iters = 0;
  cudaMemsetAsync(d, 0, sizeof(float) * N * R, h->stream);
  NDMG_CK(cudaMemcpyAsync(r, b, sizeof(float) * N * R, cudaMemcpyDeviceToDevice, h->stream));
  cudaMemsetAsync(z, 0, sizeof(float) * N * R, h->stream);
  op_vcycle<float>(h, K, r, z, true);
  if (waits_on_device(h) && (st = check_status(h)) != NDMG_OK) return st;
  if ((st = dot2<float>(h, N, b, b, r, z, bb, &S.rz)) != NDMG_OK) return st;
  std::vector<double> rz0 = S.rz;
  if ((st = cg_init(h, S, bb, bb, 2.0, &all_done)) != NDMG_OK) return st;   // relres = 1 < 2: none done
  S.rz = rz0;
  for (int i = 0; i < R; ++i) S.done[i] = bb[i] == 0.0;
  NDMG_CK(cudaMemcpyAsync(p, z, sizeof(float) * N * R, cudaMemcpyDeviceToDevice, h->stream));
  for (int it = 1; it <= maxit; ++it) {
    op_apply<float>(h, K, p, q);
    if ((st = dot2<float>(h, N, p, q, (const float*)nullptr, (const float*)nullptr, pq, nullptr)) != NDMG_OK)
      return st;
    if ((st = cg_alpha(h, S, pq, a)) != NDMG_OK) return st;
    {
      const double* da = push_coef(h, SLOT_ALPHA, a);
      Span sp(h, NDMG_K_BLAS, 6.0 * 4 * N * R);
      launch_cg_update<float>(h->stream, sm, N, da, p, q, d, r, R);
    }
    if ((st = dot2<float>(h, N, r, r, (const float*)nullptr, (const float*)nullptr, rr, nullptr)) != NDMG_OK)
      return st;
    *iters = it;
    if ((st = cg_check(h, S, rr, tol, &all_done)) != NDMG_OK) return st;
    if (all_done) return NDMG_OK;
    cudaMemsetAsync(z, 0, sizeof(float) * N * R, h->stream);
    op_vcycle<float>(h, K, r, z, true);
    if (waits_on_device(h) && (st = check_status(h)) != NDMG_OK) return st;
    if ((st = dot2<float>(h, N, r, z, q, z, rz_new, &qz)) != NDMG_OK) return st;
    for (int i = 0; i < R; ++i) {
      ab[2 * i] = 1.0;
      ab[2 * i + 1] = (S.done[i] || S.rz[i] == 0.0) ? 0.0 : -a[i] * qz[i] / S.rz[i];
      S.rz[i] = rz_new[i];
    }
    {
      const double* dab = push_coef(h, SLOT_AB, ab);
      Span sp(h, NDMG_K_BLAS, 3.0 * 4 * N * R);
      launch_axpby<float>(h->stream, sm, N, dab, z, p, R);
    }
  }
  return NDMG_OK;
}

// FP64 iterative refinement around the float PCG
int solve_ir(ndmg_t* h, const double* f, double* u, double tol, double inner_tol, int maxit, int* iters,
             double* relres) {
  const int K = h->K, R = nrhs(h);
  const int64_t N = h->lv[K].N;
  const int sm = h->sm_count;
  double* r = h->w64[0];
  float* b32 = h->w32[4];
  float* d32 = h->w32[5];
  std::vector<double> ff, rr, inv(R), rn(R);
  int st;
  *iters = 0;
  if ((st = dot2<double>(h, N, f, f, (const double*)nullptr, (const double*)nullptr, ff, nullptr)) != NDMG_OK)
    return st;
  for (int outer = 0; outer < 64; ++outer) {
    op_residual<double>(h, K, f, u, r);
    if ((st = dot2<double>(h, N, r, r, (const double*)nullptr, (const double*)nullptr, rr, nullptr)) != NDMG_OK)
      return st;
    bool all_done = true;
    double worst = 0.0;
    for (int i = 0; i < R; ++i) {
      const double nf = std::sqrt(ff[i]) > 0 ? std::sqrt(ff[i]) : 1.0;
      const double rel = std::sqrt(rr[i]) / nf;
      if (!std::isfinite(rel)) return fail(h, NDMG_BREAKDOWN, "non-finite residual");
      worst = std::fmax(worst, rel);
      const bool done = rel <= tol;
      all_done = all_done && done;
      rn[i] = done ? 0.0 : std::sqrt(rr[i]);            // converged columns get a zero correction
      inv[i] = rn[i] > 0 ? 1.0 / rn[i] : 0.0;
    }
    *relres = worst;
    if (all_done) return check_status(h);
    if (*iters >= maxit) return fail(h, NDMG_NOT_CONVERGED, "refinement reached maxit inner iterations");
    {
      const double* d = push_coef(h, SLOT_TO, inv);
      Span sp(h, NDMG_K_BLAS, 12.0 * N * R);
      launch_to_f32(h->stream, sm, N, d, r, b32, R);
    }
    int it = 0;
    if ((st = pcg32(h, b32, d32, inner_tol, maxit - *iters, &it)) != NDMG_OK) return st;
    *iters += it;
    {
      const double* d = push_coef(h, SLOT_FROM, rn);
      Span sp(h, NDMG_K_BLAS, 20.0 * N * R);
      launch_add_f32(h->stream, sm, N, d, d32, u, R);
    }
    NDMG_CK_LAUNCH();
  }
  return fail(h, NDMG_NOT_CONVERGED, "refinement stalled");
}

void free_field(ndmg_t* h) {
  for (auto& L : h->lv) {
    cudaFree(L.a64); cudaFree(L.a32); cudaFree(L.bub_gid); cudaFree(L.bubA64); cudaFree(L.bubA32);
    L.a64 = nullptr; L.a32 = nullptr; L.bub_gid = nullptr; L.bubA64 = nullptr; L.bubA32 = nullptr;
    DevGrouped* gs[4] = {&L.vtx, &L.edg[0], &L.edg[1], &L.edg[2]};
    for (DevGrouped* G : gs) {
      cudaFree(G->chunks); cudaFree(G->plist); cudaFree(G->op64); cudaFree(G->op32);
      *G = DevGrouped();
    }
    cudaFree(L.Wtc_tab); cudaFree(L.tc_off); cudaFree(L.tc_grp); cudaFree(L.tc_mask);
    L.Wtc_tab = nullptr; L.tc_off = nullptr; L.tc_grp = nullptr; L.tc_mask = nullptr;
  }
  h->field = false;
}

void free_handle(ndmg_t* h) {
  if (!h) return;
  free_field(h);
  drop_graph(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (auto& L : h->lv) {
    cudaFree(L.g64); cudaFree(L.z64); cudaFree(L.r64);
    cudaFree(L.g32); cudaFree(L.z32); cudaFree(L.r32);
    cudaFree(L.AinvT64); cudaFree(L.AinvT32); cudaFree(L.Dv64); cudaFree(L.Dv32);
    cudaFree(L.De64); cudaFree(L.De32);
    cudaFree(L.sym_v); cudaFree(L.sym_e[0]); cudaFree(L.sym_e[1]); cudaFree(L.sym_e[2]); cudaFree(L.sym_s4);
    cudaFree(L.Wtc);
    cudaFree(L.Wcell);
    cudaFree(L.Wv32);
    cudaFree(L.Wg64); cudaFree(L.WgT64); cudaFree(L.Wg32); cudaFree(L.WgT32);
  }
  cudaFree(h->Ainv0);
  for (int i = 0; i < 6; ++i) { cudaFree(h->w64[i]); cudaFree(h->w32[i]); }
  cudaFree(h->red);
  cudaFree(h->pq_red);
  cudaFree(h->umax);
  cudaFree(h->coef);
  cudaFree(h->cg);
  cudaFree(h->status);
  if (h->red_host) cudaFreeHost(h->red_host);
  if (h->coef_host) cudaFreeHost(h->coef_host);
  if (h->cg_host) cudaFreeHost(h->cg_host);
  if (h->status_host) cudaFreeHost(h->status_host);
  for (int c = 0; c < NDMG_K_COUNT; ++c)
    for (auto& pr : h->ev_used[c]) h->ev_free.push_back(pr);
  for (auto& pr : h->ev_free) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  delete h;
}

// why a mixed handle refuses a level: the rounded Gram factor no longer
// represents the vertex-patch operator (the smoother would diverge)
std::string lowp_message(int n, double lam, bool fp16) {
  char buf[320];
  std::snprintf(buf, sizeof(buf),
                "%s tensor-core operands cannot represent the vertex-patch operator of the %d^3 level "
                "(largest eigenvalue of A_p W~W~^t = %.3g > %.0g; the patch matrix is too ill-conditioned, "
                "alpha / (beta h^2) too large)%s",
                fp16 ? "fp16" : "bf16", n, lam, kTcSpectralMax,
                fp16 ? "; use NDMG_PREC_FP32" : "; use NDMG_PREC_MIXED_FP16 or NDMG_PREC_FP32");
  return buf;
}

int build_operators(ndmg_t* h) {
  const ndmg_opts& o = h->o;
  const bool fp16 = o.precision == NDMG_PREC_MIXED_FP16;
  // host work for every level first: a rejected coefficient leaves the
  // device operators untouched
  std::vector<LocalOps> all(h->K + 1);
  std::vector<double> inv;
  try {
    for (int k = h->K; k >= 1; --k) {
      DevLevel& L = h->lv[k];
      build_local_ops(L.n, o.L, o.alpha, o.beta, &all[k], o.subdomain);
      if (mixed(h) && o.subdomain == 2) {
        const double lam =
            tc_operand_spectral_max(all[k].Wv.data(), box_matrix(Box{{4, 4, 4}}, L.h, o.alpha, o.beta), fp16);
        if (!(lam <= kTcSpectralMax)) return fail(h, NDMG_INVALID_ARG, lowp_message(L.n, lam, fp16));
      }
    }
    inv = coarse_inverse(h->lv[0].n, o.L, o.alpha, o.beta);
  } catch (const std::exception& ex) {
    return fail(h, NDMG_INVALID_ARG, ex.what());
  }
  for (int k = 1; k <= h->K; ++k) {
    DevLevel& L = h->lv[k];
    const LocalOps& ops = all[k];
    if (o.subdomain == 4) {  // 108 x 108 interior solves
      NDMG_CK(upload_dense64(&L.AinvT64, ops.AinvT, 108));
      NDMG_CK(upload_sym(&L.sym_s4, &L.sym_s4_words, subdomain4_family(L.n), ops.AinvT));
    }
    else NDMG_CK(upload(&L.AinvT64, ops.AinvT));
    NDMG_CK(upload(&L.AinvT32, ops.AinvT));
    if (o.subdomain == 4) {
      // Gram factor (1176 x 312) and its transpose for k_patch_gram
      std::vector<double> WT(ops.Wv.size());
      for (int e = 0; e < ops.mV; ++e)
        for (int c = 0; c < ops.nG; ++c) WT[(size_t)c * ops.mV + e] = ops.Wv[(size_t)e * ops.nG + c];
      NDMG_CK(upload(&L.Wg64, ops.Wv));
      NDMG_CK(upload(&L.WgT64, WT));
      NDMG_CK(upload(&L.Wg32, ops.Wv));
      NDMG_CK(upload(&L.WgT32, WT));
      continue;
    }
    NDMG_CK(upload_dense64(&L.Dv64, ops.Dv, 108));
    NDMG_CK(upload_sym(&L.sym_v, &L.sym_v_words, vertex_family(L.n), ops.Dv));
    for (int d = 0; d < 3; ++d) NDMG_CK(upload_sym(&L.sym_e[d], &L.sym_e_words[d], edge_family(L.n, d), ops.De[d]));
    NDMG_CK(upload(&L.Dv32, ops.Dv));
    NDMG_CK(upload(&L.Wv32, ops.Wv));
    std::vector<double> de;
    for (int d = 0; d < 3; ++d) de.insert(de.end(), ops.De[d].begin(), ops.De[d].end());
    NDMG_CK(upload_dense64(&L.De64, de, 42));
    NDMG_CK(upload(&L.De32, de));
    if (mixed(h)) {
      cudaError_t e = upload_tc_operand(&L.Wtc, ops.Wv, fp16);
      if (e != cudaSuccess) return cuda_fail(h, e, "upload_tc_operand");
      const std::vector<uint8_t> img = tc_cell_image(ops.Wv, fp16);
      if (!L.Wcell) NDMG_CK(cudaMalloc(&L.Wcell, img.size()));
      NDMG_CK(cudaMemcpy(L.Wcell, img.data(), img.size(), cudaMemcpyHostToDevice));
    }
  }
  NDMG_CK(upload(&h->Ainv0, inv));
  for (auto& L : h->lv) {
    L.cK = o.alpha * L.h;
    L.cM = o.beta * L.h * L.h * L.h;
  }
  return NDMG_OK;
}

// Most distinct local problems one family may have on one level (each one
// is factored on the host).
constexpr int kMaxFieldGroups = 8192;

cudaError_t upload_grouped(DevGrouped* G, const GroupedFamily& g) {
  std::vector<int> plist, chunks;
  group_chunks(g, patch_group_size(), &plist, &chunks);
  G->nchunks = (int)(chunks.size() / 4);
  cudaError_t e = upload_fresh(&G->plist, plist);
  if (e == cudaSuccess) e = upload_fresh((int**)&G->chunks, chunks);
  if (e == cudaSuccess) e = upload_fresh(&G->op64, g.op);
  if (e == cudaSuccess) e = upload_fresh(&G->op32, g.op);
  return e;
}

// Coefficient per hexahedron (cells: n^3 finest-level values): the fields of
// every level (mean coarsening), grouped local operators, tensor-core images
// and brick lists, the coarsest inverse.  Host work first (it may reject the
// field), device uploads after.
int build_field_operators(ndmg_t* h, const double* cells) {
  const ndmg_opts& o = h->o;
  const int K = h->K;
  const bool edge = edge_smoother(h);
  std::vector<std::vector<double>> fld(K + 1);
  const size_t nf = (size_t)o.n * o.n * o.n;
  fld[K].assign(cells, cells + nf);
  for (int k = K; k >= 1; --k) fld[k - 1] = coarsen_cells(fld[k], h->lv[k].n);
  std::vector<FieldOps> ops(K + 1);
  std::vector<double> inv0;
  try {
    // finest first: the level with the most distinct local problems rejects a field soonest
    const int lowp = mixed(h) && !edge ? (o.precision == NDMG_PREC_MIXED_FP16 ? 2 : 1) : 0;
    for (int k = K; k >= 1; --k) {
      build_field_ops(h->lv[k].n, o.L, fld[k], o.beta, edge, kMaxFieldGroups, &ops[k], lowp);
      if (lowp && !(ops[k].vtx.tc_spectral <= kTcSpectralMax))
        return fail(h, NDMG_INVALID_ARG, lowp_message(h->lv[k].n, ops[k].vtx.tc_spectral, lowp == 2));
    }
    inv0 = coarse_inverse_cells(h->lv[0].n, o.L, fld[0], o.beta);
  } catch (const std::exception& ex) {
    return fail(h, NDMG_INVALID_ARG, ex.what());
  }
  free_field(h);
  cudaError_t e = cudaSuccess;
  for (int k = 0; k <= K && e == cudaSuccess; ++k) {
    DevLevel& L = h->lv[k];
    e = upload_fresh(&L.a64, fld[k]);
    if (e == cudaSuccess) e = upload_fresh(&L.a32, fld[k]);
    if (k == 0 || e != cudaSuccess) continue;
    const FieldOps& F = ops[k];
    e = upload_fresh(&L.bub_gid, F.bub.gid);
    if (e == cudaSuccess) e = upload_fresh(&L.bubA64, F.bub.op);
    if (e == cudaSuccess) e = upload_fresh(&L.bubA32, F.bub.op);
    if (edge) {
      for (int d = 0; d < 3 && e == cudaSuccess; ++d) e = upload_grouped(&L.edg[d], F.edge[d]);
      continue;
    }
    if (e == cudaSuccess) e = upload_grouped(&L.vtx, F.vtx);
    if (e == cudaSuccess && mixed(h)) {
      std::vector<int> off, grp;
      std::vector<uint32_t> mask;
      tc_brick_groups(L.n, F.vtx.gid, &off, &grp, &mask);
      e = upload_fresh((uint8_t**)&L.Wtc_tab,
                       tc_images(F.vtx.W, F.vtx.ngroups, o.precision == NDMG_PREC_MIXED_FP16));
      if (e == cudaSuccess) e = upload_fresh(&L.tc_off, off);
      if (e == cudaSuccess) e = upload_fresh(&L.tc_grp, grp);
      if (e == cudaSuccess) e = upload_fresh((uint32_t**)&L.tc_mask, mask);
    }
  }
  if (e == cudaSuccess) {
    cudaFree(h->Ainv0);
    h->Ainv0 = nullptr;
    e = upload(&h->Ainv0, inv0);
  }
  if (e != cudaSuccess) {
    free_field(h);
    return cuda_fail(h, e, "coefficient field upload");
  }
  h->field = true;
  for (auto& L : h->lv) {
    L.cK = L.h;  // the coefficients live in the field stencil
    L.cM = o.beta * L.h * L.h * L.h;
  }
  return NDMG_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int ndmg_opts_default(ndmg_opts* o) {
  if (!o) return NDMG_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->n = 8;
  o->n_coarsest = 2;
  o->L = 1.0;
  o->alpha = 1.0;
  o->beta = 1.0;
  o->smoother = NDMG_SMOOTHER_VERTEX;
  o->eta = 1.0 / 9.0;
  o->m = 2;
  o->precision = NDMG_PREC_FP64;
  o->nrhs = 1;
  o->stream = nullptr;
  o->subdomain = 2;
  return NDMG_OK;
}

int ndmg_create(const ndmg_opts* o, ndmg_t** out) {
  if (!out) return NDMG_INVALID_ARG;
  *out = nullptr;
  if (!o) return NDMG_INVALID_ARG;
  if (o->n < 2 || o->n_coarsest < 2 || o->n < o->n_coarsest) return NDMG_INVALID_ARG;
  if (!(o->L > 0) || !(o->alpha > 0) || !(o->beta > 0) || o->m < 1 || o->nrhs < 1) return NDMG_INVALID_ARG;
  if (o->nrhs > 4096) return NDMG_INVALID_ARG;
  if (o->smoother != NDMG_SMOOTHER_VERTEX && o->smoother != NDMG_SMOOTHER_EDGE) return NDMG_INVALID_ARG;
  const int sub = o->subdomain == 0 ? 2 : o->subdomain;
  if (sub != 2 && sub != 4) return NDMG_INVALID_ARG;
  if (sub == 4 && (o->smoother != NDMG_SMOOTHER_VERTEX || o->n_coarsest % 2 != 0)) return NDMG_INVALID_ARG;
  if (o->precision < NDMG_PREC_FP64 || o->precision > NDMG_PREC_FP32) return NDMG_INVALID_ARG;
  if (edges(o->n_coarsest) > 4096) return NDMG_INVALID_ARG;   // dense coarsest inverse
  // 32-bit edge offsets within one right-hand side (stencil, tensor-core
  // smoother): 3 n (n-1)^2 < 2^32
  if (o->n > 1024) return NDMG_INVALID_ARG;
  int K = 0;
  for (int n = o->n; n > o->n_coarsest; n /= 2, ++K)
    if (n % 2) return NDMG_INVALID_ARG;
  if ((o->n_coarsest << K) != o->n) return NDMG_INVALID_ARG;

  ndmg_t* h = new (std::nothrow) ndmg_handle();
  if (!h) return NDMG_OUT_OF_MEMORY;
  h->o = *o;
  if (!(h->o.eta > 0)) h->o.eta = h->o.smoother == NDMG_SMOOTHER_EDGE ? 1.0 / 13.0 : 1.0 / 9.0;
  if (h->o.subdomain == 0) h->o.subdomain = 2;
  h->stream = (cudaStream_t)o->stream;
  h->K = K;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    free_handle(h);
    return NDMG_CUDA_ERROR;
  }
  if (mixed(h)) {
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10) {  // tcgen05 needs a Blackwell datacenter part
      free_handle(h);
      return NDMG_INVALID_ARG;
    }
  }
  h->lv.resize(K + 1);
  cudaError_t ae = cudaSuccess;
  const int64_t R = o->nrhs;
  const bool pz = poison_workspaces();
  for (int k = 0; k <= K; ++k) {
    DevLevel& L = h->lv[k];
    L.n = o->n_coarsest << k;
    L.N = edges(L.n);
    L.h = o->L / L.n;
    L.r64 = dev_alloc<double>(L.N * R, &ae, pz);
    L.r32 = dev_alloc<float>(L.N * R, &ae, pz);
    if (k < K) {
      L.g64 = dev_alloc<double>(L.N * R, &ae, pz);
      L.z64 = dev_alloc<double>(L.N * R, &ae, pz);
      L.g32 = dev_alloc<float>(L.N * R, &ae, pz);
      L.z32 = dev_alloc<float>(L.N * R, &ae, pz);
    }
  }
  const int64_t NF = h->lv[K].N * R;
  for (int i = 0; i < 6; ++i) {
    h->w64[i] = dev_alloc<double>(NF, &ae, pz);
    h->w32[i] = dev_alloc<float>(NF, &ae, pz);
  }
  h->red = dev_alloc<double>(2 * (int64_t)reduction_blocks(h->sm_count) * R + 2 * R + 8, &ae, pz);
  {  // the finest stencil's blocks per right-hand side at its shortest z chunk (one plane), capped
    const int64_t nF = h->lv[K].n;
    h->pq_cap = std::min<int64_t>(16384, ((nF + 31) / 32) * ((nF + 7) / 8) * nF);
    h->pq_red = dev_alloc<double>(2 * h->pq_cap * R, &ae, pz);
  }
  h->umax = dev_alloc<unsigned long long>(R, &ae, pz);
  h->coef = dev_alloc<double>(4 * 2 * R, &ae, pz);
  h->cg = dev_alloc<double>(8 * R, &ae, pz);
  h->status = dev_alloc<int>(4, &ae);
  if (ae == cudaSuccess) ae = cudaMallocHost((void**)&h->red_host, (2 * R + 8) * sizeof(double));
  if (ae == cudaSuccess) ae = cudaMallocHost((void**)&h->coef_host, 4 * 2 * R * sizeof(double));
  if (ae == cudaSuccess) ae = cudaMallocHost((void**)&h->cg_host, 3 * R * sizeof(double));
  if (ae == cudaSuccess) ae = cudaMallocHost((void**)&h->status_host, 4 * sizeof(int));
  if (ae == cudaSuccess) ae = cudaMemset(h->status, 0, 4 * sizeof(int));
  if (ae == cudaSuccess) ae = prepare_stencil<double>();
  if (ae == cudaSuccess) ae = prepare_stencil<float>();
  if (ae == cudaSuccess) ae = prepare_vertex_dense<double>();
  if (ae == cudaSuccess) ae = prepare_patch_sym();
  if (ae == cudaSuccess) ae = prepare_smooth_direct();
  if (ae == cudaSuccess) ae = prepare_smooth_sym32();
  if (ae == cudaSuccess) ae = prepare_vertex_dense<float>();
  if (ae == cudaSuccess && h->o.subdomain == 4) ae = prepare_patch_gram<double>();
  if (ae == cudaSuccess && h->o.subdomain == 4) ae = prepare_patch_gram<float>();
  if (ae == cudaSuccess && mixed(h)) ae = prepare_tc_patch();
  if (ae == cudaSuccess && mixed(h)) ae = prepare_tc_cell();
  // the smallest levels in one cluster launch: levels 1 .. Kc with n <= 16
  // (constant coefficient, vertex smoother, subdomain 2, coarsest <= 4^3)
  if (ae == cudaSuccess && h->o.smoother == NDMG_SMOOTHER_VERTEX && h->o.subdomain == 2 && h->lv[0].N <= 108) {
    int Kc = 0;
    while (Kc + 1 <= K && Kc + 1 <= kCoarseMaxLevels && h->lv[Kc + 1].n <= kCoarseMaxN) ++Kc;
    if (Kc > 0) {
      ae = prepare_coarse_cycle();
      if (ae == cudaSuccess) {
        h->coarse_grid = coarse_cycle_grid(h->sm_count, Kc);
        h->Kc = h->coarse_grid > 0 ? Kc : 0;
      }
    }
  }
  if (ae == cudaSuccess) ae = prepare_stencil_field<double>();
  if (ae == cudaSuccess) ae = prepare_stencil_field<float>();
  if (ae == cudaSuccess) ae = prepare_patch_grouped<double>();
  if (ae == cudaSuccess) ae = prepare_patch_grouped<float>();
  if (ae != cudaSuccess) {
    free_handle(h);
    return ae == cudaErrorMemoryAllocation ? NDMG_OUT_OF_MEMORY : NDMG_CUDA_ERROR;
  }
  int st = build_operators(h);
  if (st != NDMG_OK) {
    std::fprintf(stderr, "ndmg_create: %s\n", h->err.c_str());
    free_handle(h);
    return st;
  }
  *out = h;
  return NDMG_OK;
}

int ndmg_destroy(ndmg_t* h) {
  if (h) cudaStreamSynchronize(h->stream);
  free_handle(h);
  return NDMG_OK;
}

const char* ndmg_last_error(const ndmg_t* h) { return h ? h->err.c_str() : "null handle"; }

int ndmg_set_alpha(ndmg_t* h, double alpha) {
  if (!h) return NDMG_INVALID_ARG;
  if (!(alpha > 0)) return fail(h, NDMG_INVALID_ARG, "alpha must be > 0");
  NDMG_CK(cudaStreamSynchronize(h->stream));
  drop_graph(h);  // the coefficients are captured in the graph's launches
  const double old = h->o.alpha;
  const bool had_field = h->field;
  h->o.alpha = alpha;
  h->field = false;             // build_operators rebuilds the constant-coefficient operators
  const int st = build_operators(h);
  if (st != NDMG_OK) {          // rejected on the host: the previous operators stay
    h->o.alpha = old;
    h->field = had_field;
    return st;
  }
  free_field(h);
  return NDMG_OK;
}

int ndmg_set_alpha_field(ndmg_t* h, const double* alpha_cells) {
  if (!h) return NDMG_INVALID_ARG;
  if (!alpha_cells) return fail(h, NDMG_INVALID_ARG, "null coefficient field");
  if (h->o.subdomain != 2) return fail(h, NDMG_INVALID_ARG, "a coefficient field needs subdomain size 2");
  const size_t nf = (size_t)h->o.n * h->o.n * h->o.n;
  for (size_t c = 0; c < nf; ++c)
    if (!(alpha_cells[c] > 0) || !std::isfinite(alpha_cells[c]))
      return fail(h, NDMG_INVALID_ARG, "coefficients must be finite and > 0");
  NDMG_CK(cudaStreamSynchronize(h->stream));
  drop_graph(h);
  const int st = build_field_operators(h, alpha_cells);
  if (st != NDMG_OK && !h->field) {
    // the handle keeps working with its constant coefficient
    const std::string msg = h->err;
    free_field(h);
    build_operators(h);
    h->err = msg;
  }
  return st;
}

int ndmg_grad_alpha_field(ndmg_t* h, const double* lambda, const double* u, double* out) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_ptrs(h, {lambda, u, out}))) return st;
  const int K = h->K, R = nrhs(h);
  DevLevel& L = h->lv[K];
  {
    Span sp(h, NDMG_K_STENCIL, (16.0 * L.N + 8.0 * L.n * L.n * L.n) * R);
    launch_grad_cells(h->stream, h->sm_count, L.n, L.h, lambda, u, out, R);
  }
  NDMG_CK_LAUNCH();
  return NDMG_OK;
}

// launches timed per candidate (small levels run near the launch rate, where
// a handful of launches is noise)
constexpr int kTuneReps = 20;

int ndmg_autotune(ndmg_t* h, int32_t* choices) {
  if (!h) return NDMG_INVALID_ARG;
  NDMG_CK(cudaStreamSynchronize(h->stream));
  drop_graph(h);  // the graph holds the launch shapes
  const int R = nrhs(h);
  const int64_t NF = h->lv[h->K].N * R;
  NDMG_CK(cudaMemsetAsync(h->w32[0], 0, sizeof(float) * NF, h->stream));
  NDMG_CK(cudaMemsetAsync(h->w32[1], 0, sizeof(float) * NF, h->stream));
  NDMG_CK(cudaMemsetAsync(h->w64[0], 0, sizeof(double) * NF, h->stream));
  NDMG_CK(cudaMemsetAsync(h->w64[1], 0, sizeof(double) * NF, h->stream));
  cudaEvent_t e0, e1;
  NDMG_CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(h, NDMG_CUDA_ERROR, "cudaEventCreate");
  }
  int st = NDMG_OK;
  for (int k = 0; k <= h->K && st == NDMG_OK; ++k) {
    DevLevel& L = h->lv[k];
    for (int t = 0; t < 2 && st == NDMG_OK; ++t) {
      float best = 0.f;
      int best_kz = 0;
      for (int kz = 1; kz <= L.n && st == NDMG_OK; kz *= 2) {
        if ((int64_t)((L.n + kz - 1) / kz) * R > 65535) continue;  // grid z: chunks x right-hand sides
        L.kz[t] = kz;
        auto run = [&] {
          if (t == 0) stencil<float>(h, k, L.cK, L.cM, h->w32[0], h->w32[1], h->w32[2]);
          else stencil<double>(h, k, L.cK, L.cM, h->w64[0], h->w64[1], h->w64[2]);
        };
        run();  // warm-up
        run();
        cudaEventRecord(e0, h->stream);
        for (int rep = 0; rep < kTuneReps; ++rep) run();
        cudaEventRecord(e1, h->stream);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          st = fail(h, NDMG_CUDA_ERROR, "autotune timing");
          break;
        }
        if (best_kz == 0 || ms < best) {
          best = ms;
          best_kz = kz;
        }
      }
      L.kz[t] = best_kz;
      if (choices) choices[3 * k + t] = best_kz;
    }
  }
  // MIXED modes, vertex smoother: tensor-core kernel or FP32 CUDA-core kernels
  // per level (small levels have too few bricks to fill the GPU)
  const bool tc_choice = mixed(h) && !edge_smoother(h) && h->o.subdomain == 2;
  // (the tensor-core kernel also for each number of cell layers per work
  // item: 0 = its own balance model, then powers of two up to n_k / 2)
  auto time_smoother = [&](int k, float* ms) -> int {
    op_smoother<float>(h, k, h->w32[0], h->w32[1]);  // warm-up
    cudaEventRecord(e0, h->stream);
    for (int rep = 0; rep < kTuneReps; ++rep) op_smoother<float>(h, k, h->w32[0], h->w32[1]);
    cudaEventRecord(e1, h->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      return fail(h, NDMG_CUDA_ERROR, "autotune timing");
    return NDMG_OK;
  };
  for (int k = 1; k <= h->K && st == NDMG_OK && tc_choice; ++k) {
    DevLevel& L = h->lv[k];
    float t_cell = 0.f, t_brick = 0.f, t_cc = 0.f;
    int best_z = 0;
    L.tc = true;
    L.tc_kind = 2;
    for (int zl = 0; zl <= L.n / 2 && st == NDMG_OK; zl = zl == 0 ? 1 : 2 * zl) {
      L.zlen = zl;
      float ms = 0.f;
      st = time_smoother(k, &ms);
      if (st == NDMG_OK && (zl == 0 || ms < t_cell)) {
        t_cell = ms;
        best_z = zl;
      }
    }
    L.zlen = best_z;
    L.tc_kind = 1;
    if (st == NDMG_OK) st = time_smoother(k, &t_brick);
    L.tc = false;
    if (st == NDMG_OK) st = time_smoother(k, &t_cc);
    L.tc = !(t_cc < t_cell && t_cc < t_brick);
    L.tc_kind = t_cell < t_brick ? 2 : 1;
  }
  for (int k = 1; k <= h->K && choices; ++k) {
    const DevLevel& L = h->lv[k];
    choices[3 * k + 2] = mixed(h) && L.tc ? L.tc_kind : 0;
  }
  // the small levels: one cluster launch or the separate launches
  if (st == NDMG_OK && h->Kc > 0 && !h->field) {
    const int kc = h->Kc;
    // the cycle's right-hand side and solution on level kc: that level's
    // own vectors, or, when kc is the finest level (every level n <= 16),
    // which has no float solution vector of its own, the float work vectors
    // (finest-level size, zeroed above)
    const float* gc = kc < h->K ? h->lv[kc].r32 : h->w32[0];
    float* zc = kc < h->K ? h->lv[kc].z32 : h->w32[1];
    float t_on = 0.f, t_off = 0.f;
    for (int v = 0; v < 2 && st == NDMG_OK; ++v) {
      h->coarse_on = v == 0;
      auto cycle = [&] {
        cudaMemsetAsync(zc, 0, sizeof(float) * h->lv[kc].N * R, h->stream);
        op_vcycle<float>(h, kc, gc, zc, true);
      };
      cycle();
      cudaEventRecord(e0, h->stream);
      for (int rep = 0; rep < kTuneReps; ++rep) cycle();
      cudaEventRecord(e1, h->stream);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        st = fail(h, NDMG_CUDA_ERROR, "autotune timing");
      (v == 0 ? t_on : t_off) = ms;
    }
    h->coarse_on = !(t_off < t_on);
  }
  if (choices) choices[2] = coarse_cycle_on(h, h->Kc) ? 1 : 0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == NDMG_OK && cudaGetLastError() != cudaSuccess) st = fail(h, NDMG_CUDA_ERROR, "autotune launch");
  if (st == NDMG_OK && waits_on_device(h)) st = check_status(h);
  return st;
}

int ndmg_select_smoother(ndmg_t* h, int32_t level, int32_t kind) {
  if (!h) return NDMG_INVALID_ARG;
  if (kind < 0 || kind > 2) return fail(h, NDMG_INVALID_ARG, "kind must be 0, 1 or 2");
  if (level < -1 || level > h->K) return fail(h, NDMG_INVALID_ARG, "level out of range");
  if (level == 0) {   // the small levels: one cluster launch (1) or separate launches (0)
    if (kind == 2) return fail(h, NDMG_INVALID_ARG, "level 0 takes kind 0 or 1");
    NDMG_CK(cudaStreamSynchronize(h->stream));
    if (int st = collect_graph(h)) return st;
    drop_graph(h);
    h->coarse_on = kind == 1;
    return NDMG_OK;
  }
  if (kind > 0 && (!mixed(h) || edge_smoother(h) || h->o.subdomain != 2))
    return fail(h, NDMG_INVALID_ARG, "tensor-core smoothers need a MIXED handle with the vertex smoother, subdomain 2");
  NDMG_CK(cudaStreamSynchronize(h->stream));
  if (int st = collect_graph(h)) return st;
  drop_graph(h);   // the graph holds the launches
  for (int k = 1; k <= h->K; ++k) {
    if (level != -1 && k != level) continue;
    h->lv[k].tc = kind > 0;
    if (kind > 0) h->lv[k].tc_kind = kind;
  }
  return NDMG_OK;
}

int ndmg_set_launch_shapes(ndmg_t* h, const int32_t* choices) {
  if (!h || !choices) return NDMG_INVALID_ARG;
  const int R = nrhs(h);
  const bool tc_ok = mixed(h) && !edge_smoother(h) && h->o.subdomain == 2;
  for (int k = 0; k <= h->K; ++k) {
    const int n = h->lv[k].n;
    for (int t = 0; t < 2; ++t) {
      const int kz = choices[3 * k + t];
      if (kz < 0 || kz > n || (kz > 0 && (int64_t)((n + kz - 1) / kz) * R > 65535))
        return fail(h, NDMG_INVALID_ARG, "planes per CTA out of range for a level");
    }
    const int kind = choices[3 * k + 2];
    if (k == 0 && (kind < 0 || kind > 1 || (kind == 1 && !(h->Kc > 0 && h->coarse_grid > 0 && !h->field))))
      return fail(h, NDMG_INVALID_ARG, "entry 2 must be 0, or 1 where the handle has levels n <= 16 for one launch");
    if (k > 0 && (kind < 0 || kind > 2 || (kind > 0 && !tc_ok)))
      return fail(h, NDMG_INVALID_ARG, "smoother kind out of range for the handle");
  }
  NDMG_CK(cudaStreamSynchronize(h->stream));
  if (int st = collect_graph(h)) return st;
  drop_graph(h);  // the graph holds the launch shapes
  for (int k = 0; k <= h->K; ++k) {
    DevLevel& L = h->lv[k];
    L.kz[0] = choices[3 * k];
    L.kz[1] = choices[3 * k + 1];
    if (k > 0 && tc_ok) {
      L.tc = choices[3 * k + 2] > 0;
      if (L.tc) L.tc_kind = choices[3 * k + 2];
      L.zlen = 0;
    }
  }
  h->coarse_on = choices[2] == 1;
  return NDMG_OK;
}

int ndmg_num_levels(const ndmg_t* h, int32_t* out) {
  if (!h || !out) return NDMG_INVALID_ARG;
  *out = h->K + 1;
  return NDMG_OK;
}

int ndmg_num_dofs(const ndmg_t* h, int32_t level, int64_t* out) {
  if (!h || !out) return NDMG_INVALID_ARG;
  if (level == -1) level = h->K;
  if (level < 0 || level > h->K) return NDMG_INVALID_ARG;
  *out = h->lv[level].N;
  return NDMG_OK;
}

int ndmg_apply(ndmg_t* h, int32_t level, int32_t dtype, const void* x, void* y) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_level(h, level, false)) || (st = check_dtype(h, dtype)) || (st = check_ptrs(h, {x, y}))) return st;
  if (dtype == NDMG_F64) op_apply<double>(h, level, (const double*)x, (double*)y);
  else op_apply<float>(h, level, (const float*)x, (float*)y);
  NDMG_CK_LAUNCH();
  return NDMG_OK;
}

int ndmg_residual(ndmg_t* h, int32_t level, int32_t dtype, const void* g, const void* z, void* r) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_level(h, level, false)) || (st = check_dtype(h, dtype)) || (st = check_ptrs(h, {g, z, r}))) return st;
  if (dtype == NDMG_F64) op_residual<double>(h, level, (const double*)g, (const double*)z, (double*)r);
  else op_residual<float>(h, level, (const float*)g, (const float*)z, (float*)r);
  NDMG_CK_LAUNCH();
  return NDMG_OK;
}

int ndmg_pencil(ndmg_t* h, int32_t level, int32_t dtype, double a, double b, const void* g, const void* x, void* y) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_level(h, level, false)) || (st = check_dtype(h, dtype)) || (st = check_ptrs(h, {x, y}))) return st;
  if (g && (st = check_ptrs(h, {g}))) return st;
  if (x == y) return fail(h, NDMG_INVALID_ARG, "y must not alias x");
  if (!std::isfinite(a) || !std::isfinite(b)) return fail(h, NDMG_INVALID_ARG, "a and b must be finite");
  if (dtype == NDMG_F64) op_pencil<double>(h, level, a, b, (const double*)g, (const double*)x, (double*)y);
  else op_pencil<float>(h, level, a, b, (const float*)g, (const float*)x, (float*)y);
  NDMG_CK_LAUNCH();
  return NDMG_OK;
}

int ndmg_axpby(ndmg_t* h, int32_t level, int32_t dtype, double a, const void* x, double b, void* y) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_level(h, level, false)) || (st = check_dtype(h, dtype)) || (st = check_ptrs(h, {x, y}))) return st;
  if (!std::isfinite(a) || !std::isfinite(b)) return fail(h, NDMG_INVALID_ARG, "a and b must be finite");
  const int64_t N = h->lv[level].N * nrhs(h);
  {
    Span sp(h, NDMG_K_BLAS, (b == 0.0 ? 2.0 : 3.0) * (dtype == NDMG_F64 ? 8 : 4) * N);
    if (dtype == NDMG_F64) launch_axpby_scalar<double>(h->stream, h->sm_count, N, a, (const double*)x, b, (double*)y);
    else launch_axpby_scalar<float>(h->stream, h->sm_count, N, a, (const float*)x, b, (float*)y);
  }
  NDMG_CK_LAUNCH();
  return NDMG_OK;
}

int ndmg_smooth(ndmg_t* h, int32_t level, int32_t dtype, const void* g, void* z, int32_t steps) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_level(h, level, true)) || (st = check_dtype(h, dtype)) || (st = check_ptrs(h, {g, z}))) return st;
  if (steps < 0) return fail(h, NDMG_INVALID_ARG, "steps must be >= 0");
  if (dtype == NDMG_F64) op_smooth_steps<double>(h, level, (const double*)g, (double*)z, steps);
  else op_smooth_steps<float>(h, level, (const float*)g, (float*)z, steps);
  NDMG_CK_LAUNCH();
  return dtype == NDMG_F32 && waits_on_device(h) ? check_status(h) : NDMG_OK;
}

int ndmg_restrict(ndmg_t* h, int32_t level, int32_t dtype, const void* r_fine, void* g_coarse) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_level(h, level, true)) || (st = check_dtype(h, dtype)) || (st = check_ptrs(h, {r_fine, g_coarse})))
    return st;
  Span sp(h, NDMG_K_RESTRICT, (dtype == NDMG_F64 ? 8.0 : 4.0) * (h->lv[level].N + h->lv[level - 1].N) * nrhs(h));
  if (dtype == NDMG_F64)
    launch_restrict<double>(h->stream, h->sm_count, h->lv[level].n, (const double*)r_fine, (double*)g_coarse, nrhs(h));
  else
    launch_restrict<float>(h->stream, h->sm_count, h->lv[level].n, (const float*)r_fine, (float*)g_coarse, nrhs(h));
  NDMG_CK_LAUNCH();
  return NDMG_OK;
}

int ndmg_prolong_add(ndmg_t* h, int32_t level, int32_t dtype, const void* z_coarse, void* z_fine) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_level(h, level, true)) || (st = check_dtype(h, dtype)) || (st = check_ptrs(h, {z_coarse, z_fine})))
    return st;
  Span sp(h, NDMG_K_PROLONG, (dtype == NDMG_F64 ? 8.0 : 4.0) * (2 * h->lv[level].N + h->lv[level - 1].N) * nrhs(h));
  if (dtype == NDMG_F64)
    launch_prolong_add<double>(h->stream, h->sm_count, h->lv[level].n, (const double*)z_coarse, (double*)z_fine,
                               nrhs(h));
  else
    launch_prolong_add<float>(h->stream, h->sm_count, h->lv[level].n, (const float*)z_coarse, (float*)z_fine,
                              nrhs(h));
  NDMG_CK_LAUNCH();
  return NDMG_OK;
}

int ndmg_coarse_solve(ndmg_t* h, int32_t dtype, const void* g, void* z) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_dtype(h, dtype)) || (st = check_ptrs(h, {g, z}))) return st;
  Span sp(h, NDMG_K_COARSE, 8.0 * h->lv[0].N * (h->lv[0].N + 2) * nrhs(h));
  if (dtype == NDMG_F64)
    launch_coarse<double>(h->stream, (int)h->lv[0].N, h->Ainv0, (const double*)g, (double*)z, nrhs(h));
  else
    launch_coarse<float>(h->stream, (int)h->lv[0].N, h->Ainv0, (const float*)g, (float*)z, nrhs(h));
  NDMG_CK_LAUNCH();
  return NDMG_OK;
}

int ndmg_vcycle(ndmg_t* h, int32_t dtype, const void* g, void* z) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_dtype(h, dtype)) || (st = check_ptrs(h, {g, z}))) return st;
  if (dtype == NDMG_F64) op_vcycle<double>(h, h->K, (const double*)g, (double*)z);
  else op_vcycle<float>(h, h->K, (const float*)g, (float*)z);
  NDMG_CK_LAUNCH();
  return dtype == NDMG_F32 && waits_on_device(h) ? check_status(h) : NDMG_OK;
}

int ndmg_solve(ndmg_t* h, const double* f, double* u, double tol, int32_t maxit, int32_t* iters, double* relres) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_ptrs(h, {f, u}))) return st;
  if (!(tol > 0) || maxit < 0) return fail(h, NDMG_INVALID_ARG, "tol must be > 0 and maxit >= 0");
  int it = 0;
  double rr = 0.0;
  if (h->o.precision == NDMG_PREC_FP64) st = pcg64(h, f, u, tol, maxit, &it, &rr);
  else st = pcg_mixed(h, f, u, tol, maxit, &it, &rr);
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return st;
}

int ndmg_solve_ir(ndmg_t* h, const double* f, double* u, double tol, double inner_tol, int32_t maxit,
                  int32_t* iters, double* relres) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_ptrs(h, {f, u}))) return st;
  if (!(tol > 0) || !(inner_tol > 0) || !(inner_tol < 1) || maxit < 0)
    return fail(h, NDMG_INVALID_ARG, "need tol > 0, 0 < inner_tol < 1, maxit >= 0");
  int it = 0;
  double rr = 0.0;
  st = solve_ir(h, f, u, tol, inner_tol, maxit, &it, &rr);
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return st;
}

int ndmg_solve_host(ndmg_t* h, const double* f_host, double* u_host, double tol, int32_t maxit, int32_t* iters,
                    double* relres) {
  if (!h) return NDMG_INVALID_ARG;
  if (!f_host || !u_host) return fail(h, NDMG_INVALID_ARG, "null host buffer");
  const int64_t N = h->lv[h->K].N * nrhs(h);
  double* f = h->w64[4];
  double* u = h->w64[5];
  NDMG_CK(cudaMemcpyAsync(f, f_host, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
  NDMG_CK(cudaMemcpyAsync(u, u_host, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
  int st = ndmg_solve(h, f, u, tol, maxit, iters, relres);
  if (st != NDMG_OK && st != NDMG_NOT_CONVERGED) return st;
  NDMG_CK(cudaMemcpyAsync(u_host, u, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
  NDMG_CK(cudaStreamSynchronize(h->stream));
  return st;
}

int ndmg_vcycle_iterate(ndmg_t* h, const double* f, double* u, double tol, int32_t maxit, int32_t* cycles,
                        double* relres) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_ptrs(h, {f, u}))) return st;
  const int K = h->K, R = nrhs(h);
  const int64_t N = h->lv[K].N;
  double* r = h->w64[0];
  std::vector<double> ff, rr;
  if ((st = dot2<double>(h, N, f, f, (const double*)nullptr, (const double*)nullptr, ff, nullptr)) != NDMG_OK)
    return st;
  for (int c = 0;; ++c) {
    op_residual<double>(h, K, f, u, r);
    if ((st = dot2<double>(h, N, r, r, (const double*)nullptr, (const double*)nullptr, rr, nullptr)) != NDMG_OK)
      return st;
    double worst = 0.0;
    for (int i = 0; i < R; ++i) {
      const double nf = std::sqrt(ff[i]) > 0 ? std::sqrt(ff[i]) : 1.0;
      const double rel = std::sqrt(rr[i]) / nf;
      if (!std::isfinite(rel)) return fail(h, NDMG_BREAKDOWN, "non-finite residual");
      worst = std::fmax(worst, rel);
    }
    if (relres) *relres = worst;
    if (cycles) *cycles = c;
    if (worst <= tol) return NDMG_OK;
    if (c >= maxit) return fail(h, NDMG_NOT_CONVERGED, "V-cycle iteration reached maxit");
    op_vcycle<double>(h, K, f, u);
  }
}

int ndmg_grad_alpha(ndmg_t* h, const double* lambda, const double* u, double* out) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_ptrs(h, {lambda, u}))) return st;
  if (!out) return fail(h, NDMG_INVALID_ARG, "null output");
  const int K = h->K, R = nrhs(h);
  DevLevel& L = h->lv[K];
  // one fused pass: circulations of lambda and u per cell, face-mass pairs,
  // FP64 block sums (reads lambda and u; each edge from its 4 cells via L1)
  const int nb = reduction_blocks(h->sm_count);
  double* sums = h->red + 2 * (int64_t)nb * R;
  {
    Span sp(h, NDMG_K_BLAS, 16.0 * L.N * R, 2);
    launch_grad_alpha_sum(h->stream, h->sm_count, L.n, L.h, lambda, u, h->field ? L.a64 : nullptr, h->red, sums, R);
  }
  std::vector<double> v;
  if ((st = read_sums(h, sums, v, nullptr, false)) != NDMG_OK) return st;
  for (int i = 0; i < R; ++i) out[i] = v[i];
  return NDMG_OK;
}

int ndmg_dot(ndmg_t* h, int32_t level, int32_t dtype, const void* x, const void* y, double* out) {
  if (!h) return NDMG_INVALID_ARG;
  int st;
  if ((st = check_level(h, level, false)) || (st = check_dtype(h, dtype)) || (st = check_ptrs(h, {x, y}))) return st;
  if (!out) return fail(h, NDMG_INVALID_ARG, "null output");
  const int64_t N = h->lv[level].N;
  std::vector<double> v;
  if (dtype == NDMG_F64)
    st = dot2<double>(h, N, (const double*)x, (const double*)y, (const double*)nullptr, (const double*)nullptr, v,
                      nullptr);
  else
    st = dot2<float>(h, N, (const float*)x, (const float*)y, (const float*)nullptr, (const float*)nullptr, v, nullptr);
  if (st != NDMG_OK) return st;
  for (int i = 0; i < nrhs(h); ++i) out[i] = v[i];
  return NDMG_OK;
}

int ndmg_trace_enable(ndmg_t* h, int32_t kernel_class, int32_t on) {
  if (!h) return NDMG_INVALID_ARG;
  if (kernel_class < 0 || kernel_class >= NDMG_K_COUNT) return fail(h, NDMG_INVALID_ARG, "bad kernel class");
  if (h->trace_on[kernel_class] != (on != 0)) {
    NDMG_CK(cudaStreamSynchronize(h->stream));
    if (int st = collect_graph(h)) return st;
    drop_graph(h);  // recaptured with (or without) this class's events
  }
  h->trace_on[kernel_class] = on != 0;
  return NDMG_OK;
}

int ndmg_use_graphs(ndmg_t* h, int32_t on) {
  if (!h) return NDMG_INVALID_ARG;
  NDMG_CK(cudaStreamSynchronize(h->stream));
  if (int st = collect_graph(h)) return st;
  drop_graph(h);
  h->use_graphs = on != 0;
  return NDMG_OK;
}

int ndmg_trace_read(ndmg_t* h, int32_t kernel_class, int64_t* launches, double* ms, double* units) {
  if (!h) return NDMG_INVALID_ARG;
  if (kernel_class < 0 || kernel_class >= NDMG_K_COUNT) return fail(h, NDMG_INVALID_ARG, "bad kernel class");
  NDMG_CK(cudaStreamSynchronize(h->stream));
  if (int st = collect_graph(h)) return st;
  double total = h->trace_ms_graph[kernel_class];
  h->trace_ms_graph[kernel_class] = 0.0;
  for (auto& pr : h->ev_used[kernel_class]) {
    float t = 0.f;
    NDMG_CK(cudaEventElapsedTime(&t, pr.first, pr.second));
    total += t;
    h->ev_free.push_back(pr);
  }
  h->ev_used[kernel_class].clear();
  if (launches) *launches = h->trace_launches[kernel_class];
  if (ms) *ms = total;
  if (units) *units = h->trace_units[kernel_class];
  h->trace_launches[kernel_class] = 0;
  h->trace_units[kernel_class] = 0.0;
  return NDMG_OK;
}

int ndmg_inject_status(ndmg_t* h, int32_t code) {
  if (!h) return NDMG_INVALID_ARG;
  if (code < 0) return fail(h, NDMG_INVALID_ARG, "status code must be >= 0");
  NDMG_CK(cudaStreamSynchronize(h->stream));
  *h->status_host = code;
  NDMG_CK(cudaMemcpyAsync(h->status, h->status_host, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  NDMG_CK(cudaStreamSynchronize(h->stream));
  return NDMG_OK;
}

int ndmg_counters(const ndmg_t* h, int64_t* launches, int64_t* vcycles) {
  if (!h) return NDMG_INVALID_ARG;
  if (launches) *launches = h->launch_total;
  if (vcycles) *vcycles = h->vcycle_total;
  return NDMG_OK;
}

}  // extern "C"
