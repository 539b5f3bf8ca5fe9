// Internal declarations of libndmg (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/ndmg.h"

namespace ndmg {

// Interior edges of a box of bx*by*bz cells (the canonical layout of
// ndmg.h with per-axis extents), N = bx(by-1)(bz-1) + (bx-1)by(bz-1) + (bx-1)(by-1)bz.
struct Box {
  int b[3];
  int64_t count(int d) const {
    int64_t c = 1;
    for (int a = 0; a < 3; ++a) c *= (a == d) ? b[a] : (b[a] - 1);
    return c;
  }
  int64_t size() const { return count(0) + count(1) + count(2); }
  // index of edge (d, i, j, k) in box coordinates or -1 if not interior
  int64_t index(int d, int i, int j, int k) const;
};

// ---- host-side local operators (setup.cpp) ---------------------------------
struct LocalOps {
  int n;                      // cells per side on this level
  double h;
  int s = 2;                  // subdomain size (cells per side of a subdomain)
  int mT = 6;                 // interior edges of one subdomain: 3 s (s-1)^2
  int mV = 108;               // edges of one vertex patch: 3 (2s) (2s-1)^2
  int nG = 60;                // interface edges of one vertex patch
  std::vector<double> AinvT;  // mT x mT inverse of the interior-space matrix A_T
  std::vector<double> Dv;     // mV x mV J_V A_V^{-1} J_V^t (patch-local order; s = 2 only)
  std::vector<double> Wv;     // mV x nG Gram factor, J_V A_V^{-1} J_V^t = Wv Wv^t
  std::vector<double> De[3];  // 42x42 J_E A_E^{-1} J_E^t for coarse edges along x, y, z (s = 2)
};

// Dense assembled matrix of a box with Dirichlet (interior-edge) DOFs for
// a(w,v) = alpha (curl w, curl v) + beta (w, v) on cubes of side h.
std::vector<double> box_matrix(const Box& box, double h, double alpha, double beta);
// The same with a curl-curl coefficient per cell of the box (acell: one value
// per cell, x fastest).
std::vector<double> box_matrix_cells(const Box& box, double h, const double* acell, double beta);
// J_D A_D^{-1} J_D^t of the discrete-harmonic space of a box of cells split
// into s x s x s subdomains, from the box's assembled matrix Ap: dense D
// (optional) and Gram factor W (np x n_interface).
void patch_operator(const Box& pb, int s, const std::vector<double>& Ap, std::vector<double>* D,
                    std::vector<double>* W, int* n_interface);
// Vertex-patch operator and Gram factor, interior-space inverse for level n
// with subdomains of s x s x s cells (s = 2: the coarse elements).
void build_local_ops(int n, double L, double alpha, double beta, LocalOps* out, int s = 2);
// Inverse of the coarsest operator (n0^3 box).
std::vector<double> coarse_inverse(int n0, double L, double alpha, double beta);
// In-place Cholesky of an SPD matrix (lower), returns false if not SPD.
bool cholesky(std::vector<double>& a, int n);
std::vector<double> spd_inverse(const std::vector<double>& a, int n, bool* ok);

// ---- curl-curl coefficient constant per hexahedron (field.cpp) ---------------
// One family of local problems on one level (interior spaces, vertex or edge
// patches), grouped by the coefficients of the cells each one covers.
struct GroupedFamily {
  int nloc = 0;             // edges of one local problem
  int nG = 0;               // interface edges (vertex patches)
  int ngroups = 0;
  std::vector<int> gid;     // group of every member, in family order
  std::vector<double> op;   // ngroups x nloc x nloc: A_T^{-1} (interior) or J A^{-1} J^t (patches)
  std::vector<double> W;    // ngroups x nloc x nG Gram factors (vertex patches)
  double tc_spectral = 0.0; // largest eigenvalue of A_p W~ W~^t over the groups (rounded operands; 0 unchecked)
};
struct FieldOps {
  GroupedFamily bub;        // interior spaces of the coarse elements
  GroupedFamily vtx;        // vertex patches (vertex-based smoother)
  GroupedFamily edge[3];    // edge patches along x, y, z (edge-based smoother)
};
// mean of the 8 fine coefficients of every coarse hexahedron (n -> n/2)
std::vector<double> coarsen_cells(const std::vector<double>& a, int n);
// local operators of level n for cell coefficients acell (n^3, x fastest);
// throws if a family has more than max_groups distinct local problems
// lowp: 0, or the tensor-core operand type to check the vertex groups for
// (1 = bf16, 2 = fp16; sets vtx.tc_spectral)
void build_field_ops(int n, double L, const std::vector<double>& acell, double beta, bool edge, int max_groups,
                     FieldOps* out, int lowp = 0);
std::vector<double> coarse_inverse_cells(int n0, double L, const std::vector<double>& acell, double beta);
// members listed group by group (plist) and chunks {group, first, count, 0}
// of at most pb members of one group
void group_chunks(const GroupedFamily& g, int pb, std::vector<int>* plist, std::vector<int>* chunks);

// ---- device side -----------------------------------------------------------
// bits of the handle's device status word
constexpr int kStatusBreakdown = 64;     // PCG met a non-positive or non-finite curvature p^T A p

// PCG scalars on the device, R entries each (ab: 2 per right-hand side)
struct CgScalars {
  double *alpha, *ab, *sto, *sfrom, *rz, *rr, *done;
};
enum CgMode { CG_ALPHA = 0, CG_RR = 1, CG_BETA = 2, CG_BETA_FLEX = 3, CG_RZ = 4 };

// a grouped family on the device (coefficient field)
struct DevGrouped {
  int nchunks = 0;
  int4* chunks = nullptr;   // {group, first plist entry, count, 0}
  int* plist = nullptr;     // members, group by group
  double* op64 = nullptr;   // ngroups x nloc x nloc
  float* op32 = nullptr;
};

struct DevLevel {
  int n;
  int64_t N;                  // edges on this level
  double h, cK, cM;           // alpha*h, beta*h^3
  int kz[2] = {0, 0};         // stencil planes per CTA for float / double vectors (ndmg_autotune; 0 = built-in)
  bool tc = true;             // MIXED modes: vertex patches on tensor cores on this level (ndmg_autotune may
                              // pick the FP32 CUDA-core kernels where they finish sooner)
  // FP64 workspaces (coarse levels) and FP32 workspaces
  double *g64 = nullptr, *z64 = nullptr, *r64 = nullptr;
  float *g32 = nullptr, *z32 = nullptr, *r32 = nullptr;
  // local operators (levels >= 1)
  double* AinvT64 = nullptr;  // 36
  float* AinvT32 = nullptr;
  double* Dv64 = nullptr;     // 108*108
  float* Dv32 = nullptr;
  double* De64 = nullptr;     // 3 * 42*42 (edge-based smoother)
  // the FP64 dense operators in the mirror-symmetry basis (patch_sym.cu):
  // vertex patches, edge patches per direction, subdomain-4 interiors
  uint32_t* sym_v = nullptr;
  uint32_t* sym_e[3] = {nullptr, nullptr, nullptr};
  uint32_t* sym_s4 = nullptr;
  int sym_v_words = 0, sym_e_words[3] = {0, 0, 0}, sym_s4_words = 0;
  float* De32 = nullptr;
  void* Wtc = nullptr;        // tensor-core operand images (bf16/fp16), see tc kernel
  void* Wcell = nullptr;      // the same factor in the per-neighbour blocks of the cell-owned kernel (tc_cell.cu)
  float* Wv32 = nullptr;      // the Gram factor W (108 x 60, FP32) for the persistent small-level kernel
  int zlen = 0;               // cell-owned smoother: cell layers per work item (ndmg_autotune; 0 = built-in)
  int tc_kind = 1;            // tensor-core smoother: 1 brick kernel (tc_patch.cu), 2 cell-owned kernel (tc_cell.cu)
  // subdomain size 4: Gram factor of the 1176-edge vertex patches (1176 x 312)
  // and its transpose, for k_patch_gram
  double *Wg64 = nullptr, *WgT64 = nullptr;
  float *Wg32 = nullptr, *WgT32 = nullptr;
  // curl-curl coefficient per hexahedron (ndmg_set_alpha_field); cK is then h
  double* a64 = nullptr;      // n^3 cell coefficients
  float* a32 = nullptr;
  int* bub_gid = nullptr;     // group of every coarse element's interior space
  double* bubA64 = nullptr;   // 36 per group
  float* bubA32 = nullptr;
  DevGrouped vtx, edg[3];     // vertex patches; edge patches along x, y, z
  void* Wtc_tab = nullptr;    // tensor-core operand image per vertex group
  int* tc_off = nullptr;      // per brick: first entry of its group list (nbricks + 1)
  int* tc_grp = nullptr;      // per entry: group
  uint4* tc_mask = nullptr;   // per entry: the brick's rows (patches) in that group
};

}  // namespace ndmg

struct ndmg_handle {
  ndmg_opts o;
  cudaStream_t stream;
  int sm_count;
  int K;                                  // finest level index
  std::vector<ndmg::DevLevel> lv;         // lv[0] = coarsest
  double* Ainv0 = nullptr;                // coarsest inverse (FP64, N0 x N0)
  // PCG / refinement workspaces on the finest level
  double *w64[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  float *w32[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* red = nullptr;                  // reduction scratch (partials + results)
  double* pq_red = nullptr;               // the finest-level FP64 stencil's block partial sums of p.q
  int64_t pq_cap = 0;                     // ... room per right-hand side (blocks)
  double* red_host = nullptr;             // pinned mirror of the results (2 per right-hand side)
  double* coef = nullptr;                 // per-right-hand-side BLAS scalars (4 slots x 2R)
  double* coef_host = nullptr;            // pinned staging of those scalars
  double* cg = nullptr;                   // device PCG scalars (CgScalars, 8 R doubles)
  double* cg_host = nullptr;              // pinned: rr read back, done flags pushed (2 R doubles)
  int* status = nullptr;                  // device status word (timeouts)
  // the smallest levels of the float V-cycle in one cluster launch
  // (coarse_cycle.cu): levels 1 .. Kc (n <= 16) and the coarsest
  int Kc = 0;                             // 0: not available for this handle
  int coarse_grid = 0;                    // CTAs of its cluster
  bool coarse_on = false;                 // ndmg_autotune / ndmg_select_smoother may switch it on
  unsigned long long* umax = nullptr;     // per right-hand side max |u| of the fixed-point FP64 stencil
  int* status_host = nullptr;             // pinned mirror of the status word
  std::string err;
  bool field = false;                     // curl-curl coefficient per hexahedron (ndmg_set_alpha_field)
  // tracing: per kernel class, event pairs recorded around launches
  bool trace_on[NDMG_K_COUNT] = {};
  int64_t trace_launches[NDMG_K_COUNT] = {};
  double trace_units[NDMG_K_COUNT] = {};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used[NDMG_K_COUNT];
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_free;
  int64_t launch_total = 0;
  int64_t vcycle_total = 0;
  double trace_ms_graph[NDMG_K_COUNT] = {};  // elapsed time collected from graph replays
  // the float V-cycle of the mixed preconditioner (z32 = MG(K, r32, 0, m)),
  // captured once as a CUDA graph and replayed; traced launches inside it are
  // bracketed by event-record nodes whose times are collected after each replay
  struct GraphSpan {
    int cls;
    double units;
    int nlaunch;
    cudaEvent_t a, b;
  };
  bool use_graphs = true;
  bool capturing = false;
  bool graph_pending = false;               // a replay whose spans are not collected yet
  cudaGraphExec_t vgraph = nullptr;
  cudaStream_t cap_stream = nullptr;        // private stream the graph is captured on
  std::vector<GraphSpan> vgraph_spans;
  int64_t vgraph_launches = 0, vgraph_vcycles = 0;
};
