/*
 * ndmg.h -- C ABI of libndmg: V-cycle multigrid for the lowest-order
 * hexahedral Nedelec discretisation of curl(alpha curl u) + beta u = f on an
 * axis-aligned box [0,L]^3 with zero tangential trace, smoothed by the
 * nonoverlapping domain-decomposition smoothers of Oh, "Multigrid methods for
 * 3D H(curl) problems with nonoverlapping domain decomposition smoothers"
 * (arXiv 2205.05840).  One GPU (sm_103a), no CPU fallback.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Mesh.  Level k (0 = coarsest, K = finest) has n_k = n_0 * 2^k hexahedra per
 *   side, h_k = L / n_k (Sec. 3.1: uniform refinement, h_k = h_{k-1}/2).
 * DOFs.  One value per interior edge (Sec. 2, eq. NDdof: the average
 *   tangential component), N(n) = 3 n (n-1)^2, canonical order, every edge
 *   oriented along +axis:
 *     x-edge (segment i in [0,n), nodes j,k in [1,n-1]): ((k-1)(n-1)+(j-1)) n + i
 *     y-edge (node i in [1,n-1], segment j in [0,n), node k): n(n-1)^2 + ((k-1) n + j)(n-1) + (i-1)
 *     z-edge (nodes i,j in [1,n-1], segment k in [0,n)): 2n(n-1)^2 + (k(n-1) + (j-1))(n-1) + (i-1)
 *   Right-hand sides are load (dual) vectors <f_h, phi_e>.
 * Batches.  With opts.nrhs = R > 1 every vector argument holds R right-hand
 *   sides one after the other: right-hand side r is the canonical vector at
 *   offset r * N(n_k).  All R are processed by the same launches (the batch is
 *   a grid dimension of every kernel); solvers iterate them in lockstep with
 *   per-right-hand-side scalars, and scalar outputs become arrays of R.
 * Pointers.  Vector arguments are DEVICE pointers owned by the caller (for
 *   instance torch tensors), contiguous, at least 16-byte aligned, and of the
 *   element type named by the call's `dtype` (NDMG_F64 = double, NDMG_F32 =
 *   float).  Entry points whose name ends in _host take HOST pointers
 *   instead.  Scalar outputs are host pointers, written before return.
 * Streams.  Work is queued on the handle's stream (opts.stream, NULL = the
 *   legacy default stream).  Calls that return scalars synchronise that
 *   stream; the others return as soon as the work is queued.
 * Errors.  Every call returns an ndmg_status.  On failure the handle keeps a
 *   message (ndmg_last_error); nothing is allocated or freed by a failing
 *   call except by ndmg_create, which releases what it built.  Invalid
 *   arguments are detected on the host before any launch.
 * Threads.  A handle may be used by one host thread at a time.
 */
#ifndef NDMG_H
#define NDMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ndmg_status {
  NDMG_OK = 0,
  NDMG_INVALID_ARG = 1,
  NDMG_CUDA_ERROR = 2,
  NDMG_OUT_OF_MEMORY = 3,
  NDMG_NOT_CONVERGED = 4,
  NDMG_BREAKDOWN = 5,     /* PCG: non-positive or non-finite curvature / NaN */
  NDMG_DEVICE_TIMEOUT = 6 /* a bounded device-side wait gave up; results invalid */
} ndmg_status;

typedef enum ndmg_dtype { NDMG_F64 = 0, NDMG_F32 = 1 } ndmg_dtype;

/* Smoother of Sec. 3.2. */
typedef enum ndmg_smoother {
  NDMG_SMOOTHER_VERTEX = 0, /* eq. (Preconditioner P), default eta 1/9 */
  NDMG_SMOOTHER_EDGE = 1    /* eq. (Preconditioner E), default eta 1/13; CUDA cores in every precision mode */
} ndmg_smoother;

/* Arithmetic of the V-cycle.  FP64: everything in double.  MIXED_BF16 /
 * MIXED_FP16: the inner V-cycle runs on float vectors (stencil, transfers,
 * interior solves in FP32) with the vertex-patch solves on tensor cores in
 * bf16 / fp16 with FP32 accumulation (the product that forms the patch
 * output, W t, with W's high and low-order bf16 / fp16 parts; t = W^t r with
 * single-rounded operands); residuals of the outer refinement loop, PCG
 * inner products and the coarsest solve stay in double. */
typedef enum ndmg_precision {
  NDMG_PREC_FP64 = 0,
  NDMG_PREC_MIXED_BF16 = 1,
  NDMG_PREC_MIXED_FP16 = 2,
  NDMG_PREC_FP32 = 3 /* float V-cycle, patch solves on CUDA cores (FP32) */
} ndmg_precision;

typedef struct ndmg_opts {
  int32_t n;          /* hexahedra per side on the finest level, <= 1024; even unless n == n_coarsest */
  int32_t n_coarsest; /* hexahedra per side on the coarsest level (paper: 2); n = n_coarsest * 2^K */
  double L;           /* box side length, > 0 */
  double alpha;       /* curl-curl coefficient, > 0 (eq. 1) */
  double beta;        /* mass coefficient, > 0 (1 in eq. 1; eps + sigma dt/2 in eq. Maxwell timestep) */
  int32_t smoother;   /* ndmg_smoother */
  double eta;         /* damping factor; <= 0 selects the paper's value (1/9 vertex, 1/13 edge) */
  int32_t m;          /* pre- and post-smoothing steps per level (Fig. 1), >= 1 */
  int32_t precision;  /* ndmg_precision */
  int32_t nrhs;       /* right-hand sides per call, >= 1 */
  void* stream;       /* cudaStream_t, NULL = legacy default stream */
  int32_t subdomain;  /* cells per side of a smoother subdomain: 2 (Sec. 3.2: the coarse elements) or 4
                         (4x4x4 blocks, 1176-edge vertex patches; vertex smoother only; every smoothed
                         level a multiple of 4, i.e. n_coarsest even); 0 selects 2 */
} ndmg_opts;

typedef struct ndmg_handle ndmg_t;

/* Fill *o with defaults: n = 8, n_coarsest = 2, L = 1, alpha = beta = 1,
 * vertex smoother with eta = 1/9, m = 2, FP64, nrhs = 1, default stream. */
int ndmg_opts_default(ndmg_opts* o);

/* Build the level hierarchy of Sec. 3.1 and every local operator of Sec. 3.2
 * for the options in *o: the interior-space matrix A_T of eq. (ATDef) and its
 * inverse, the vertex-space operator J_V A_V^{-1} J_V^t of eq. (AVDef) as a
 * dense 108x108 matrix and as a Gram factor W (108x60, W W^t = the same
 * operator), and the coarsest inverse A_0^{-1} (Fig. 1, k = 0).  Allocates all
 * device workspaces.  *out receives the handle (NULL on failure).  Errors:
 * INVALID_ARG (bad sizes, alpha/beta/L <= 0, nrhs < 1, unsupported smoother;
 * MIXED precision whose rounded Gram factor W~ cannot carry the vertex-patch
 * operator: largest eigenvalue of A_p W~W~^t above 16, which bf16 operands can
 * reach from alpha / (beta h^2) ~ 3e5 on (23 at 4.1e5 on a 64^3 level; the value
 * also depends on the rounded factor's bit patterns, 7.3 there on 32^3 and
 * 128^3) and fp16 ones only beyond ~2.5e7 -- the smoother would diverge; the
 * message names the level), OUT_OF_MEMORY, CUDA_ERROR.
 * Debugging aid: with the environment variable NDMG_POISON_WORKSPACES=1 set
 * when the handle is created, every device workspace starts as all-one bytes
 * (NaN in float and double), so a read of an entry nothing has written shows
 * up as NaN results. */
int ndmg_create(const ndmg_opts* o, ndmg_t** out);

/* Free every resource of the handle (NULL is accepted). */
int ndmg_destroy(ndmg_t* h);

/* Message of the last failing call on this handle ("" if none); owned by the
 * handle, valid until the next call on it. */
const char* ndmg_last_error(const ndmg_t* h);

/* Rebuild the local operators for a new alpha (eq. 1), keeping all buffers
 * (a coefficient field, if one was set, is dropped).  Errors: INVALID_ARG
 * (alpha <= 0, or a MIXED handle whose operands cannot carry the new operator,
 * as for ndmg_create; the handle keeps its previous coefficient), CUDA_ERROR. */
int ndmg_set_alpha(ndmg_t* h, double alpha);

/* Curl-curl coefficient constant on every hexahedron (eq. 1 with a
 * piecewise-constant alpha; the jumping coefficients named in the concluding
 * remarks).  alpha_cells: HOST pointer to n^3 doubles for the finest level,
 * cell (i, j, k) (the hexahedron [i,i+1]x[j,j+1]x[k,k+1] h) at (k n + j) n + i,
 * each finite and > 0; copied, not kept.  Coarser levels take the mean of the 8
 * fine coefficients in each coarse hexahedron (rediscretisation).  The
 * smoother keeps the paper's spaces (Sec. 3.2) with the local matrices of the
 * actual coefficients: subdomains and patches whose cells carry bitwise equal
 * coefficients share one factorisation, so the number of distinct local
 * problems per family and level is limited to 8192 (piecewise-constant
 * materials stay far below; a field that differs in every cell does not).
 * With a field set, K in ndmg_pencil and ndmg_grad_alpha is the
 * coefficient-weighted curl-curl matrix sum_T alpha_T K_T (so A = K + beta M,
 * and ndmg_grad_alpha gives the derivative for alpha scaled by a common
 * factor, at factor 1); ndmg_set_alpha returns to a constant coefficient.
 * Subdomain size 2 only.  Synchronises the handle's stream; host set-up time
 * grows with the number of distinct local problems (one 108-edge Schur
 * complement each).  Errors: INVALID_ARG (NULL, non-positive or non-finite
 * values, subdomain size 4, too many distinct local problems, a MIXED handle
 * whose operands cannot carry some vertex-patch operator of the field (as for
 * ndmg_create); the handle keeps its previous coefficients), OUT_OF_MEMORY,
 * CUDA_ERROR. */
int ndmg_set_alpha_field(ndmg_t* h, const double* alpha_cells);

/* Per-hexahedron derivative of a loss L(u(f, alpha)) with respect to the
 * coefficient of each finest-level cell, given the adjoint lambda (A lambda =
 * dL/du): out[r n^3 + cell] = -lambda_r^T K_T u_r, with K_T the alpha-free
 * curl-curl element matrix of that cell (its derivative of a(., .) = sum_T
 * alpha_T (curl ., curl .)_T + beta (., .)).  Valid with or without a field.
 * lambda, u: double device vectors of the finest level [x nrhs]; out: double
 * device array of n^3 x nrhs, caller-owned; all 16-byte aligned.
 * Asynchronous on the handle's stream.  Errors: INVALID_ARG, CUDA_ERROR. */
int ndmg_grad_alpha_field(ndmg_t* h, const double* lambda, const double* u, double* out);

/* Autotuner for the kernels' launch shapes (no counterpart in the paper):
 * for every level and both vector types (float, double) it times the
 * streaming stencil for each power-of-two number of z-planes per CTA (1 ..
 * n_k; twenty launches each, CUDA events on the handle's stream, with the
 * handle's nrhs) and keeps the fastest; every choice computes bitwise the same
 * result.  On MIXED handles with the vertex smoother it also times, per level,
 * the two tensor-core smoothers (per brick of 128 vertex patches; cell-owned
 * rows, for every number of cell layers per work item: its own balance model,
 * then 1, 2, 4, ... n_k / 2) and the FP32 CUDA-core smoother (small levels
 * have too little work to fill the GPU), and keeps the fastest; the FP32
 * kernels are at least as accurate.  It then times the levels n <= 16 in one
 * launch of a thread-block cluster against separate launches per step and
 * keeps the faster.
 * Synchronises the stream, overwrites the handle's solver workspaces and
 * drops a captured V-cycle graph.  choices: NULL or a host array of 3 (K+1)
 * ints, level-major: [3k] planes per CTA for float, [3k+1] for double, [3k+2]
 * (k >= 1) the smoother of level k: 0 CUDA cores, 1 tensor cores per brick,
 * 2 tensor cores on cell-owned rows; [2] (the coarsest level has no smoother)
 * 1 when the levels n <= 16 run in one cluster launch, else 0.
 * Errors: INVALID_ARG, CUDA_ERROR, DEVICE_TIMEOUT. */
int ndmg_autotune(ndmg_t* h, int32_t* choices);

/* Applies launch shapes chosen earlier (by ndmg_autotune on a handle of the
 * same size, levels, precision and nrhs, on the same kind of GPU) without
 * timing anything: choices is a host array of 3 (K+1) ints in ndmg_autotune's
 * format (planes per CTA 0 = the built-in choice; the cell-owned smoother, if
 * chosen, takes its built-in number of cell layers per work item).  The
 * planes per CTA leave results bitwise unchanged; the smoother kinds differ
 * in summation order only.  Synchronises the stream and drops
 * a captured V-cycle graph.  Errors: INVALID_ARG (an entry out of range for
 * the handle; nothing is changed), CUDA_ERROR. */
int ndmg_set_launch_shapes(ndmg_t* h, const int32_t* choices);

/* Chooses the smoother kernel of a level by hand (what ndmg_autotune decides
 * by timing): kind 0 FP32 CUDA cores, 1 tensor cores per brick of 128 vertex
 * patches, 2 tensor cores on cell-owned rows (both tensor-core kernels compute
 * eq. (Preconditioner P); the brick kernel forms the patch outputs with W's
 * high and low-order parts, the cell-owned kernel with its single rounding,
 * and they differ in how the overlapping patch outputs are summed).  level: 1 .. K, or -1 for every
 * level.  Kinds 1 and 2 need a MIXED handle with the vertex smoother and
 * subdomain size 2.  level 0 instead selects how float V-cycles run the
 * levels n <= 16 (when the handle has them): kind 1 in one launch of a
 * thread-block cluster, 0 (the default) in separate launches per step.
 * Synchronises the stream and drops a captured V-cycle graph.
 * Errors: INVALID_ARG, CUDA_ERROR. */
int ndmg_select_smoother(ndmg_t* h, int32_t level, int32_t kind);

/* Number of levels K+1. */
int ndmg_num_levels(const ndmg_t* h, int32_t* out);

/* N(n_k) for level k (k = -1 means the finest). */
int ndmg_num_dofs(const ndmg_t* h, int32_t level, int64_t* out);

/* y = A_k x (Sec. 2: <A_h w, v> = a(w, v)), matrix-free.  x, y: N(n_k) [x nrhs]. */
int ndmg_apply(ndmg_t* h, int32_t level, int32_t dtype, const void* x, void* y);

/* y = g + (a K_k + b M_k) x: any member of the pencil whose (alpha, beta)
 * member is A_k (eq. 1: a(w,v) = alpha (curl w, curl v) + beta (w, v)), with
 * K_k the alpha-free curl-curl matrix and M_k the mass matrix of level k.
 * An implicit Maxwell step (Sec. 1, eq. (Maxwell timestep)) forms its
 * right-hand side from the two previous time levels with two such calls.
 * g may be NULL (then y = (a K_k + b M_k) x).  x, g, y: N(n_k) [x nrhs]
 * vectors of dtype, caller-owned device memory, 16-byte aligned; y may alias
 * g but not x.  Asynchronous on the handle's stream.  Errors: INVALID_ARG
 * (level, dtype, pointers, aliasing, non-finite a or b), CUDA_ERROR. */
int ndmg_pencil(ndmg_t* h, int32_t level, int32_t dtype, double a, double b, const void* g, const void* x, void* y);

/* y = a x + b y elementwise over all nrhs right-hand sides of level k (y is
 * not read when b = 0).  No counterpart in the paper: the vector update that
 * time-stepping drivers need between solves (warm-start extrapolation).
 * Pointers as for ndmg_pencil; x may alias y.  Errors: INVALID_ARG, CUDA_ERROR. */
int ndmg_axpby(ndmg_t* h, int32_t level, int32_t dtype, double a, const void* x, double b, void* y);

/* r = g - A_k z. */
int ndmg_residual(ndmg_t* h, int32_t level, int32_t dtype, const void* g, const void* z, void* r);

/* `steps` smoothing steps z <- z + M_k^{-1} (g - A_k z) (Fig. 1) on level
 * k >= 1, with M_k^{-1} the smoother of eq. (Preconditioner P).  dtype F64
 * uses the FP64 patch operator; dtype F32 uses the handle's precision mode
 * (tensor-core patch solves in the MIXED modes, FP32 CUDA cores otherwise). */
int ndmg_smooth(ndmg_t* h, int32_t level, int32_t dtype, const void* g, void* z, int32_t steps);

/* g_c = I_k^{k-1} r_f (eq. F2C), level k >= 1: r_f on level k, g_c on k-1. */
int ndmg_restrict(ndmg_t* h, int32_t level, int32_t dtype, const void* r_fine, void* g_coarse);

/* z_f += I_{k-1}^k z_c (Sec. 3.1, natural injection), level k >= 1. */
int ndmg_prolong_add(ndmg_t* h, int32_t level, int32_t dtype, const void* z_coarse, void* z_fine);

/* z = A_0^{-1} g on the coarsest level (Fig. 1, k = 0). */
int ndmg_coarse_solve(ndmg_t* h, int32_t dtype, const void* g, void* z);

/* z <- MG(K, g, z, m) on the finest level (Fig. 1), z in/out. */
int ndmg_vcycle(ndmg_t* h, int32_t dtype, const void* g, void* z);

/* Solve A_K u = f to ||f - A u||_2 <= tol ||f||_2 with conjugate gradients
 * preconditioned by one V-cycle MG(K, ., 0, m) (symmetric: Remark 6).  FP64
 * handles run FP64 PCG.  MIXED / FP32 handles run the same FP64 PCG (FP64
 * vectors, residuals and inner products, flexible beta) with the float
 * V-cycle as preconditioner: 2^-e r with 2^(e-1) <= ||r|| < 2^e is handed
 * to the V-cycle in float and its result scaled back by 2^e in double (power
 * of two scales: both are exact exponent shifts; float results below the
 * smallest normal float flush to zero).  f, u: double device vectors, u in/out
 * (warm start).  *iters: PCG iterations (= V-cycles), *relres: final relative
 * residual in FP64 (either may be NULL).  Returns NOT_CONVERGED after maxit
 * iterations, BREAKDOWN on a non-finite residual or non-positive curvature. */
int ndmg_solve(ndmg_t* h, const double* f, double* u, double tol, int32_t maxit,
               int32_t* iters, double* relres);

/* FP64 iterative refinement (MIXED / FP32 handles): repeat r = f - A u in
 * FP64; solve A d = r / ||r|| with float PCG + float V-cycle to relative
 * inner_tol (0 < inner_tol < 1); u += ||r|| d; until ||f - A u|| <= tol ||f||.
 * maxit bounds the total inner PCG iterations (reported in *iters). */
int ndmg_solve_ir(ndmg_t* h, const double* f, double* u, double tol, double inner_tol, int32_t maxit,
                  int32_t* iters, double* relres);

/* As ndmg_solve with HOST f and u: copies f in and u out on the handle's
 * stream (pinned memory recommended) and synchronises. */
int ndmg_solve_host(ndmg_t* h, const double* f_host, double* u_host, double tol, int32_t maxit,
                    int32_t* iters, double* relres);

/* Standalone iteration u <- MG(K, f, u, m) until ||f - A u|| <= tol ||f|| or
 * maxit cycles (Sec. 5 style), FP64 vectors. */
int ndmg_vcycle_iterate(ndmg_t* h, const double* f, double* u, double tol, int32_t maxit,
                        int32_t* cycles, double* relres);

/* dL/dalpha of a loss L(u(f, alpha)) given the adjoint lambda (A lambda =
 * dL/du; A is symmetric, Remark 6): out[r] = -lambda_r^T K u_r with K the
 * alpha-free curl-curl matrix (a(w,v) = alpha (curl w, curl v) + beta (w, v));
 * with a coefficient per hexahedron K = sum_T alpha_T K_T.  One fused kernel
 * forms the face circulations of lambda and u cell by cell, pairs them through
 * the face mass and reduces in FP64 (then a finishing kernel per right-hand
 * side).  lambda, u: double device vectors on the finest level; out: host,
 * nrhs doubles (synchronises the handle's stream). */
int ndmg_grad_alpha(ndmg_t* h, const double* lambda, const double* u, double* out);

/* Graph replay of the float V-cycle inside the mixed-precision solves (no
 * counterpart in the paper; launch latency only): with on != 0 (the default)
 * the V-cycle that preconditions each FP64 iteration is captured once as a
 * CUDA graph on the handle's stream and replayed; on == 0 launches it kernel
 * by kernel.  The graph is recaptured after ndmg_set_alpha or a change of
 * ndmg_trace_enable.  Synchronises the handle's stream.  Errors: INVALID_ARG,
 * CUDA_ERROR. */
int ndmg_use_graphs(ndmg_t* h, int32_t on);

/* Inner product in FP64: out[r] = x_r^T y_r for each of the nrhs right-hand
 * sides (out: host, nrhs doubles). */
int ndmg_dot(ndmg_t* h, int32_t level, int32_t dtype, const void* x, const void* y, double* out);

/* ---- tracing (no counterpart in the paper: measurement support) --------
 * Kernel classes whose launches can be timed with CUDA events recorded on the
 * handle's stream around every launch of that class. */
typedef enum ndmg_kernel_class {
  NDMG_K_STENCIL = 0,  /* operator apply / residual */
  NDMG_K_RESTRICT = 1,
  NDMG_K_PROLONG = 2,
  NDMG_K_BUBBLE = 3,   /* interior-space solves */
  NDMG_K_PATCH = 4,    /* vertex-patch solves (CUDA-core or tensor-core kernel) */
  NDMG_K_COARSE = 5,
  NDMG_K_BLAS = 6,     /* reductions and vector updates */
  NDMG_K_COUNT = 7
} ndmg_kernel_class;

/* Switch event timing of one kernel class on (on != 0) or off. */
int ndmg_trace_enable(ndmg_t* h, int32_t kernel_class, int32_t on);

/* Synchronise, then report and reset the class's totals since the last read:
 * launches, summed device time in ms, and summed algorithmic work: bytes a
 * launch must move to or from memory (every vector read or written once) for
 * the memory-bound classes; for NDMG_K_PATCH arithmetic operations (flops) on
 * FP64 / FP32 handles and, on MIXED handles (memory-bound there), the
 * smoother's 12 bytes per edge of float vectors (read r, read and write z). */
int ndmg_trace_read(ndmg_t* h, int32_t kernel_class, int64_t* launches, double* ms, double* units);

/* Host-side fault injection for tests (no counterpart in the paper): writes
 * code (>= 0) into the handle's device status word, exactly as a tensor-core
 * kernel does when one of its bounded waits gives up.  While the word is
 * nonzero the kernels that check it (the tensor-core smoothers of MIXED
 * handles) return without doing anything; the next entry point that reads it
 * (ndmg_solve, ndmg_vcycle, ndmg_smooth on float vectors of a MIXED handle)
 * returns NDMG_DEVICE_TIMEOUT and clears it, after which the handle works as
 * before.  Synchronises the handle's stream.  Errors: INVALID_ARG, CUDA_ERROR. */
int ndmg_inject_status(ndmg_t* h, int32_t code);

/* Running totals since ndmg_create: kernels launched by this handle (all
 * classes) and V-cycles MG(K, ., ., m) performed on the finest level.  Either
 * pointer may be NULL. */
int ndmg_counters(const ndmg_t* h, int64_t* launches, int64_t* vcycles);

/* Measured FMA rate of the CUDA cores of the current device (no counterpart
 * in the paper; the roofline denominator of kernels bound by the FP64 or FP32
 * pipe): *tflops = 2 x fused multiply-adds per second of many independent
 * FMA chains (dtype NDMG_F64 or NDMG_F32), timed with CUDA events over five
 * launches of ~50 ms total at the clocks the GPU runs (nothing is locked).
 * Allocates and frees one element; synchronises the device's legacy stream.
 * Errors: INVALID_ARG, CUDA_ERROR. */
int ndmg_probe_fma_rate(int32_t dtype, double* tflops);

/* ---- allocation-free inner product (no counterpart in the paper) ---------
 * out = x^T y in FP64 for n elements of type dtype (NDMG_F64 or NDMG_F32),
 * for callers that cannot allocate device memory: code running under an
 * allocator that owns every device byte of the process, code where a
 * cudaMalloc (which may synchronise the device) is not acceptable, or code
 * that cannot create a handle (ndmg_create allocates all level workspaces).
 * No handle is needed and nothing is allocated: the partial sums live in a
 * fixed 32 KB device array inside the library, which every GPU that loads the
 * library holds until the process exits.
 *   x, y   device pointers, n elements each (caller-owned), 16-byte aligned
 *          like every vector of this library (the kernels themselves read
 *          single elements, so element alignment would be enough for them)
 *   n      0 <= n <= 67,108,864; larger n returns NDMG_INVALID_ARG (and a
 *          message on stderr) before anything is launched
 *   out    host pointer, written before return
 *   stream cudaStream_t (NULL = legacy default stream); the call queues two
 *          kernels and a copy on it and synchronises it.
 * The first call on a device looks up the device address of the array (with
 * that device current) and keeps it for the device's current CUDA context; a
 * call in another context of the device (after cudaDeviceReset, or under a
 * non-primary context) looks it up again.  Make that first call before any
 * stream capture.  All
 * calls share the one array, so calls that overlap on the GPU (other host
 * threads, other streams) race and give wrong results; serialise them.  The
 * array keeps the last call's contents; each call overwrites every slot it
 * reads.  Errors: INVALID_ARG (bad dtype, NULL or misaligned pointers, n out
 * of range), CUDA_ERROR. */
int ndmg_dot_noalloc(int32_t dtype, const void* x, const void* y, int64_t n, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NDMG_H */
