/*
 * vk.h -- C ABI of a single-GPU (GB300, sm_103a) matrix-full Vanka multigrid solver for the
 * Taylor-Hood (P_k, P_{k-1}) discretization of the Stokes equations on triangles.
 *
 * Method: Rafiei and MacLachlan, "Achieving h- and p-robust monolithic multigrid solvers for the
 * Stokes equations", arXiv 2409.14222.
 *   - Stokes problem and weak form:            Sec. 2, Eqs. (Stokes1), (VariationalStokesa/b)
 *   - Taylor-Hood on triangles (Case 1):       Sec. 3
 *   - saddle-point system per level, nested hierarchy, canonical transfers, R = P^T,
 *     Chebyshev-accelerated additive relaxation on [lambda/4, 1.1 lambda]:  Sec. 3
 *   - additive subspace correction:            Algorithm 1 (Sec. 3.1)
 *   - vertex / edge / cell composite patches:  Sec. 3.1
 *   - matrix-full patch extraction (ASMPatchPC-style): Sec. 3.1, last paragraph
 *   - FGMRES outer solver, zero initial guess, relative reduction, at most 100 iterations: Sec. 3, Sec. 4
 *
 * Conventions (all calls):
 *   - Vectors are FP64, length ndof of the level, in the canonical DoF order: velocity node-major
 *     (DoF 2*node + component, node = b*(kN+1) + a for the lattice point (a/(kN), b/(kN))), then the
 *     pressure lattice ((k-1)N+1)^2 at offset 2*(kN+1)^2.
 *   - Pointers named *_dev are device pointers owned by the caller; they must stay valid until the
 *     work queued on `stream` has finished.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *   - Every call returns a status code (VK_OK = 0).  On error, vk_last_error() gives a message for
 *     the calling thread.  A hierarchy is not thread-safe; distinct hierarchies are independent.
 *   - Level 0 is the coarsest mesh; level nlevels-1 the finest.
 */
#ifndef VK_H
#define VK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VK_ABI_VERSION 1

/* ---- status codes ---------------------------------------------------------------------------- */
#define VK_OK 0
#define VK_ERR_ARG 1            /* invalid argument or call not valid for this hierarchy        */
#define VK_ERR_NO_MEMORY 2      /* device allocation failed (allocator returned NULL)           */
#define VK_ERR_SINGULAR 3       /* zero pivot in a patch matrix or in the coarse bordered matrix */
#define VK_ERR_NONFINITE 4      /* NaN or Inf in a right-hand side or residual                  */
#define VK_ERR_NOT_CONVERGED 5  /* FGMRES reached maxit; x and info are still valid             */
#define VK_ERR_TIMEOUT 6        /* a bounded device-side wait expired                           */
#define VK_ERR_CUDA 7           /* CUDA runtime error                                           */
#define VK_ERR_INTERNAL 8
#define VK_ERR_CANCELLED 9      /* a queued solve request was cancelled, or the service stopped   */

/* ---- options ----------------------------------------------------------------------------------- */
#define VK_WEIGHTS_PLAIN 0         /* Algorithm 1 with w_i = gamma_i = identity (a plain sum)       */
#define VK_WEIGHTS_MULTIPLICITY 1  /* each DoF's correction divided by the number of its patches    */

#define VK_PREC_F64 0  /* patch inverses stored and applied in FP64                                  */
#define VK_PREC_F32 1  /* patch inverses stored in FP32, applied with FP32 products, FP64 vectors    */
#define VK_PREC_F64E 2 /* patch inverses stored as FP32 (hi, lo) pairs (48 significant bits) and
                          applied in FP32-pair arithmetic (exact product split + TwoSum accumulation)
                          on the FP32 pipes; relative accuracy about 1e-13; FP64 vectors            */

#define VK_BATCH_NONE 0  /* no multi-right-hand-side support (vk_solve_batch refused)             */
#define VK_BATCH_BF16 1  /* vk_solve_batch: FP32 V-cycle, BF16 scaled patch inverses on tensor cores */
#define VK_BATCH_FP16 2  /* vk_solve_batch: FP32 V-cycle, FP16 scaled patch inverses on tensor cores */

#define VK_ENGINE_TCGEN05 0   /* vk_solve_batch patch solves: tcgen05.mma, TMEM accumulators, TMA loads   */
#define VK_ENGINE_MMA_SYNC 1  /* the same contraction with warp-level mma.sync m16n8k16 (for comparison) */

#define VK_ASSEMBLY_MATRIX_FULL 0  /* patch matrices gathered from the assembled CSR matrix (ASMPatchPC, Sec. 3.1) */
#define VK_ASSEMBLY_MATRIX_FREE 1  /* patch matrices assembled from element matrices per patch (PCPATCH, Sec. 3.1) */

#define VK_CSR_A 0  /* level matrix script-A_l with Dirichlet identity rows and zeroed columns      */
#define VK_CSR_P 1  /* prolongation from level l-1 to level l (ndof_l x ndof_{l-1})                 */
#define VK_CSR_R 2  /* restriction R = P^T (ndof_{l-1} x ndof_l)                                     */

#define VK_BC_DIRICHLET_ALL 0  /* velocity Dirichlet condition on the whole boundary (Eq. StokesDirichletNoSlip) */

#define VK_CELL_TRIANGLE 0  /* Taylor-Hood (P_k, P_{k-1}) on triangles (Case 1 of Sec. 3), 2 <= k <= 4       */
#define VK_CELL_QUAD 1      /* Taylor-Hood (Q_k, Q_{k-1}) on quadrilaterals (Case 2 of Sec. 3), 2 <= k <= 4:
                               the same lattice DoF layout; vertex patches, and for k >= 3 edge and
                               cell patches (Sec. 3.1; interior sizes 51 / 99, 57, 33 / 163, 92, 54 for
                               k = 2 / 3 / 4); the N x N squares of the unit square                */
#define VK_CELL_BDM 2       /* (BDM_k, dP_{k-1}) on triangles (Case 3 of Sec. 3), 1 <= k <= 5: H(div)-
                               conforming velocity, discontinuous pressure, the interior-penalty form
                               of Eq. (DiscontBilinearForm) with alpha = (k+1)(k+2), u . n = 0 imposed on
                               the boundary-edge DoFs, extended cell patches (Sec. 3.1; interior size
                               4 (k+1)(k+2) - 3 (k+1) + k (k+1) / 2: 19, 42, 74, 115, 165 for k = 1..5);
                               matrix-full patches only.  DoFs: per edge (oriented from its lower to its
                               higher vertex id, vertex id = y (N+1) + x) the normal fluxes
                               v(x_j) . rot(x_b - x_a), rot(x, y) = (y, -x), at x_j = x_a + (j+1)/(k+2)
                               (x_b - x_a); per cell the moments of the pulled-back field against
                               Nedelec's first-kind space of degree k - 1 on the reference cell (its
                               monomial basis orthogonalised in L^2 and scaled to norms in [1, 2) by
                               powers of two); per
                               cell the pressure at the equispaced P_{k-1} nodes.  Order: edge DoFs
                               (horizontal, vertical, diagonal edges, each lexicographic), then each
                               cell's interior DoFs, then each cell's pressures (lower cells, then
                               upper).  The Dirichlet rows of this discretization are the no-flux rows:
                               b there is the prescribed normal flux (zero for Eq. model_problem).  */

/* Mesh hierarchy: the unit square cut into N_coarse x N_coarse squares, each split from its top-left
 * to its bottom-right corner (Sec. 4), refined uniformly nlevels-1 times (Sec. 3).  Velocity is
 * continuous P_k, pressure continuous P_{k-1} (Case 1 of Sec. 3), 2 <= k <= 4; nu is the viscosity of
 * Eq. (Stokes1).
 *   bc:     VK_BC_DIRICHLET_ALL is the only boundary condition of the method (the paper's problem has
 *           a velocity Dirichlet condition on all of the boundary, Eqs. StokesDirichletNoSlip and
 *           model_problem); any other value is refused with VK_ERR_ARG.  The boundary VALUES are data
 *           of the right-hand side, not of the hierarchy: Dirichlet rows of the matrix are identity rows
 *           (their columns zeroed), so b's entries at the Dirichlet DoFs (vk_export_dirichlet) are the
 *           prescribed velocities and the remaining entries must already carry the lifting
 *           F - A_FB g of nonzero data (the manufactured problem of Sec. 4 is built that way).
 *   domain: {x0, x1, y0, y1} of the rectangle; the method is stated on the unit square (Sec. 4), so
 *           only {0, 1, 0, 1} is accepted (all four zero is read as that default); anything else is
 *           refused with VK_ERR_ARG. */
typedef struct vk_problem {
  int32_t N_coarse;
  int32_t nlevels;
  int32_t k;
  double nu;
  int32_t bc;
  double domain[4];
  int32_t cell;        /* VK_CELL_TRIANGLE (0, the default of a zeroed struct), VK_CELL_QUAD or
                          VK_CELL_BDM (k in 1..5 for VK_CELL_BDM)                                   */
} vk_problem;

typedef struct vk_options {
  int32_t sweeps;      /* Chebyshev steps per pre- and post-smoothing (nu in Sec. 4), >= 1          */
  int32_t weights;     /* VK_WEIGHTS_*                                                               */
  double cheb_lo;      /* Chebyshev interval [cheb_lo*lambda, cheb_hi*lambda]; 0.25 and 1.1 (Sec. 3) */
  double cheb_hi;
  int32_t eig_steps;   /* Arnoldi steps of the largest-eigenvalue estimate (10)                     */
  uint64_t eig_seed;   /* SplitMix64 seed of the Arnoldi start vector; level l uses eig_seed + l    */
  const double* lambdas; /* optional host array of nlevels values (index 0 unused); NULL = estimate */
  int32_t factor_prec; /* VK_PREC_*                                                                  */
  int32_t use_graph;   /* 1: replay each FGMRES iteration as a captured CUDA graph                  */
  int32_t host_threads;/* threads for host assembly (0 = hardware concurrency)                      */
  int32_t host_only;   /* 1: build and keep the host-side hierarchy only (export calls, no solves)  */
  int32_t max_iterations; /* FGMRES basis size allocated at setup (100, the paper's cap, Sec. 4)   */
  int32_t batch_prec;     /* VK_BATCH_*: build the multi-right-hand-side structures (needs FP64
                             factor_prec: the 16-bit inverses are rounded from the FP64 ones)     */
  int32_t batch_max_iterations; /* FGMRES basis size of vk_solve_batch per right-hand side (<= 127) */
  int32_t autotune;       /* 1: at setup, time every candidate launch shape of the patch application
                             on each smoothed level and keep the fastest (vk_apply_schedule)      */
  int32_t apply_schedule; /* -1: autotune (or the default shape when autotune = 0); >= 0: use that
                             candidate on every level (candidates are listed at vk_apply_schedule) */
  int32_t batch_engine;   /* VK_ENGINE_*: tensor-core instruction family of vk_solve_batch          */
  int32_t test_expire_wait; /* test of the bounded device waits: 1 makes the first finest-level
                               tcgen05 patch sweep after setup announce one bulk copy without
                               issuing it, so its wait expires (about 2 s), the kernel ends cleanly
                               and vk_solve_batch returns VK_ERR_TIMEOUT; later calls run normally.
                               0 (default) in normal use                                           */
  int32_t spmv_warps;     /* SELL layout of the sparse products: threads per row = the smallest of
                             1, 2, 4, 8 that gives at least this many warps per SM (default 48)    */
  int32_t batch_coarse_fp32; /* vk_solve_batch: 0 (default) keeps the coarsest-level dense solve in
                             FP64 inside the FP32 V-cycle; 1 applies an FP32 copy of the inverse   */
  int32_t test_singular_patch; /* test of the singular-patch path: >= 0 zeroes, in the copy of the
                             finest-level matrix uploaded for the patch gather only, the row of the
                             last DoF of that (canonical) finest-level patch, so its patch matrix is
                             singular and vk_setup returns VK_ERR_SINGULAR naming that patch; -1
                             (default) in normal use                                                */
  int32_t patch_assembly;  /* VK_ASSEMBLY_*: how the patch matrices are formed before they are factored.
                             MATRIX_FULL (default) extracts them from the global CSR matrix by the
                             patches' DoF lists; MATRIX_FREE assembles each one from the element
                             matrices of every cell containing one of its DoFs (redundant work on
                             overlapping patches, as the paper notes for PCPATCH).  Both sum each entry
                             over the same cells in the same order, so the patch matrices, inverses
                             and solves are bit-identical; only the setup cost differs
                             (vk_stats.setup_factor_ms)                                             */
  int32_t graph_pdl;       /* 1: the whole-solve graph's kernels are captured with programmatic
                             dependent launch (each may be launched before its predecessor has fully
                             retired, and waits for that grid's completion before touching memory);
                             if the driver refuses the capture, the graph is rebuilt without it
                             (vk_stats.graph_pdl reports which).  0 (default): ordinary launches —
                             measured on GB300 no faster at 128x128 or 512x512.  Results are identical
                             either way                                                              */
} vk_options;

/* Device memory provider.  alloc returns device memory of at least `bytes` (256-byte aligned) or
 * NULL; release frees it.  Both are called only from vk_setup / vk_destroy on the calling thread.
 * Passing NULL to vk_setup uses cudaMalloc / cudaFree. */
typedef struct vk_allocator {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*release)(void* ctx, void* ptr, void* stream);
} vk_allocator;

typedef struct vk_hierarchy vk_hierarchy;

typedef struct vk_solve_info {
  int32_t iterations;  /* FGMRES iterations (= V-cycles) performed                                 */
  int32_t converged;   /* 1 if the residual estimate reached rtol * ||b||                          */
  double res0;         /* ||b|| after projection off the constant pressure                         */
  double res_est;      /* last Givens residual estimate                                            */
  double true_res;     /* ||b - A x|| recomputed at exit                                           */
  double* history;     /* optional caller-owned host array of maxit+1 doubles: res0, then the
                          residual estimate after each iteration; NULL to skip                     */
  double solve_ms;     /* wall time of the call in milliseconds (host clock, includes the sync)    */
} vk_solve_info;

/* Fills *o with the defaults used by the paper's setting: 1 sweep, plain weights, [0.25, 1.1],
 * 10 Arnoldi steps, FP64 factors, graphs on, patch-apply autotuning on. */
void vk_default_options(vk_options* o);

/* Builds the hierarchy (Sec. 3): per level the assembled CSR saddle-point matrix (Sec. 3), the
 * canonical prolongation / restriction (Sec. 3), the composite Vanka patches (Sec. 3.1), every patch
 * matrix gathered from the CSR matrix and inverted by Gauss-Jordan elimination with partial pivoting
 * on the GPU (Sec. 3.1, matrix-full), the bordered coarsest-level inverse, and the Chebyshev
 * eigenvalue estimate of each smoothed level (Sec. 3).  Returns VK_ERR_SINGULAR if a patch or the
 * coarse bordered matrix has a zero pivot.  The hierarchy owns all device memory it allocates through
 * `alloc` (NULL = cudaMalloc); work is queued on `stream` and synchronised before return. */
int vk_setup(const vk_problem* p, const vk_options* o, const vk_allocator* alloc, void* stream,
             vk_hierarchy** out);

/* Checks a problem and options as vk_setup does (ranges, bc, domain, option values) without building
 * anything.  Returns VK_OK or VK_ERR_ARG with a message. */
int vk_check_problem(const vk_problem* p, const vk_options* o);

/* Frees the hierarchy and every device buffer it owns.  NULL is ignored. */
void vk_destroy(vk_hierarchy* h);

/* Message of the last failed call on this thread ("" if none).  Valid until the next call. */
const char* vk_last_error(void);

/* Device bytes vk_setup would allocate for (p, o).  Builds the host-side structures only (no device
 * work, no device memory): used to admit solves by HBM footprint. */
int vk_footprint(const vk_problem* p, const vk_options* o, size_t* device_bytes);

/* Sizes of one level: DoFs, velocity DoFs, nonzeros of A, number of patches and patch slots
 * (sum of patch sizes).  Any output pointer may be NULL. */
int vk_level_info(const vk_hierarchy* h, int level, int32_t* ndof, int32_t* n_u, int64_t* nnz,
                  int32_t* npatch, int64_t* nslots);

/* Device bytes this hierarchy allocated (equals vk_footprint for the same problem and options). */
int vk_device_bytes(const vk_hierarchy* h, size_t* bytes);

/* Chebyshev eigenvalue estimate lambda of level `level` (>= 1): the largest real part of the Ritz
 * values of eig_steps Arnoldi steps on M^{-1} A (Sec. 3, "standard GMRES estimation"). */
int vk_lambda(const vk_hierarchy* h, int level, double* lambda);

/* Launch shape of the patch application on level `level` (>= 1), chosen at setup.  Patches of
 * uneven size (boundary and interior vertex patches, edge and cell patches for k >= 3: Sec. 3.1) are
 * applied either in one launch (split = 0; each warp dispatches on its patch's size) or in one launch
 * per size class of ceil(n/4) (1-4, 5-10, 11-19, 20-32, 33-42; split = 1); threads per block 128 or 256;
 * per_sm = 0 launches one warp per patch, per_sm > 0 a persistent grid of per_sm blocks per SM.
 * Candidate i is split = i / 6, threads = (i / 3) % 2 ? 256 : 128, per_sm = {0, 4, 8}[i % 3]
 * (*ncand = 12 of them).  cand_us (host, *ncand doubles, may be NULL) receives each candidate's best
 * time in microseconds from the autotuner (0 if it did not run).  The corrections are bit-identical
 * for every shape. */
int vk_apply_schedule(const vk_hierarchy* h, int level, int32_t* split, int32_t* threads, int32_t* per_sm,
                      int32_t* index, double* cand_us, int32_t* ncand);

/* r = b - A_level x  (CSR SpMV residual; Algorithm 1's local right-hand sides come from it). */
int vk_residual(vk_hierarchy* h, int level, const double* b_dev, const double* x_dev, double* r_dev,
                void* stream);

/* z = M^{-1} r: one application of the additive Vanka operator of Algorithm 1 on level `level`
 * (>= 1): every patch solve delta_i = A_i^{-1} r[idx_i] is applied with the stored inverse, then the
 * weighted corrections are summed into each DoF in ascending patch order (no atomics); Dirichlet
 * DoFs get z = r.  r_dev and z_dev must not alias. */
int vk_vanka(vk_hierarchy* h, int level, const double* r_dev, double* z_dev, void* stream);

/* Same result as vk_vanka, but the call allocates no device memory: the per-slot corrections go to
 * one fixed 8 MiB device array (2^20 FP64 values) compiled into the library, instead of the buffer
 * the hierarchy allocated at setup.  For callers that must not allocate at the point of use: a
 * process whose device memory is reserved up front by another allocator, or a thread that must not
 * risk the device-wide synchronisation that cudaMalloc / cudaFree can cause.  (The paper has no
 * counterpart: this is a deployment variant of Algorithm 1's additive correction.)
 *   - Levels with more than 2^20 patch slots (sum of patch sizes, vk_level_info) get VK_ERR_ARG.
 *   - The array exists once per GPU that loads the library and lives until the process exits.
 *   - The first call on a device looks the array's device address up with that device current
 *     (cudaGetSymbolAddress); make that first call before any stream capture on that device.
 *   - All calls share the array: calls whose work overlaps on the GPU (other streams, other threads,
 *     other hierarchies) race on it and must be serialised by the caller.  Nothing in it needs to
 *     start at zero; it keeps the last call's values. */
int vk_vanka_noalloc(vk_hierarchy* h, int level, const double* r_dev, double* z_dev, void* stream);

/* `sweeps` Chebyshev steps (Sec. 3, "Relaxation") of the Vanka-preconditioned iteration for
 * A_level x = b on [cheb_lo*lambda, cheb_hi*lambda].  zero_init = 1 ignores x on input (x0 = 0). */
int vk_smooth(vk_hierarchy* h, int level, const double* b_dev, double* x_dev, int zero_init,
              void* stream);

/* r_coarse = R r_fine with R = P^T (Sec. 3), then zero at the coarse Dirichlet DoFs.
 * fine_level >= 1; r_coarse has the DoFs of fine_level - 1. */
int vk_restrict(vk_hierarchy* h, int fine_level, const double* r_fine_dev, double* r_coarse_dev,
                void* stream);

/* x_fine += P e_coarse (canonical prolongation of Sec. 3).  fine_level >= 1. */
int vk_prolong(vk_hierarchy* h, int fine_level, const double* e_coarse_dev, double* x_fine_dev,
               void* stream);

/* x = solution of the bordered coarsest system [[A_0, z], [z^T, 0]] [x; mu] = [b; 0] with
 * z = (0_u, 1_p) the constant pressure (reading: the paper does not name its coarse solver),
 * applied as a GEMV with the inverse computed at setup. */
int vk_coarse_solve(vk_hierarchy* h, const double* b_dev, double* x_dev, void* stream);

/* x = V(nu, nu)(b): one multiplicative V-cycle on the finest level with zero initial guess
 * (Sec. 3): Chebyshev/Vanka pre-smoothing, residual, restriction, recursion, prolongation,
 * post-smoothing; the coarsest level is solved by vk_coarse_solve. */
int vk_vcycle(vk_hierarchy* h, const double* b_dev, double* x_dev, void* stream);

/* Solves A x = b on the finest level with right-preconditioned unrestarted FGMRES (Sec. 3),
 * preconditioned by one V-cycle, zero initial guess, stopping when the Givens residual estimate is
 * <= rtol * ||b|| or after maxit (<= 100 is the paper's setting, Sec. 4) iterations.  b is projected
 * off the constant pressure first and every preconditioned vector is projected too, so x has zero
 * pressure mean.  Orthogonalisation: classical Gram-Schmidt applied twice.  x_dev is overwritten.
 * Returns VK_ERR_NOT_CONVERGED (with x and info valid) if maxit was reached, VK_ERR_NONFINITE if b
 * or an iterate is not finite.  `info` (host, may be NULL) is complete when the call returns. */
int vk_solve(vk_hierarchy* h, const double* b_dev, double* x_dev, double rtol, int maxit,
             vk_solve_info* info, void* stream);

/* Solves A X = B for nrhs <= 16 right-hand sides at once (B, X: device, column-major, ndof x nrhs,
 * leading dimension ldb >= ndof).  Each column is an independent FGMRES solve with the vk_solve
 * semantics in FP64 (projection, CGS2, Givens, its own convergence test and iteration count); the
 * V-cycle preconditioner runs on all columns together in FP32, with every patch solve of Algorithm 1
 * applied as a small dense product on the tensor cores (BF16 or FP16 inverses scaled per patch; with
 * FP16 each right-hand-side column is also scaled to its largest magnitude over the patch, which
 * BF16's FP32-sized exponent does not need; FP32 accumulation); the coarsest-level solve stays FP64
 * unless batch_coarse_fp32 is set.  A column's result does not depend
 * on the other columns.  Needs a hierarchy set up with batch_prec != VK_BATCH_NONE.  infos (host,
 * nrhs entries, may be NULL) receive the per-column results; histories are not recorded.
 * Returns VK_ERR_NOT_CONVERGED if a column reached maxit, VK_ERR_NONFINITE if a column diverged. */
int vk_solve_batch(vk_hierarchy* h, int nrhs, const double* B_dev, int64_t ldb, double* X_dev, double rtol,
                   int maxit, vk_solve_info* infos, void* stream);

/* vk_solve with host buffers: copies b_host (ndof doubles) to the device, solves, copies x back to
 * x_host.  Both copies are issued on `stream`; the call returns after x_host is written. */
int vk_solve_host(vk_hierarchy* h, const double* b_host, double* x_host, double rtol, int maxit,
                  vk_solve_info* info, void* stream);

/* Dimensions of CSR matrix `which` (VK_CSR_*) of a level (P and R need level >= 1). */
int vk_csr_dims(const vk_hierarchy* h, int level, int which, int32_t* nrows, int32_t* ncols,
                int64_t* nnz);

/* Copies CSR matrix `which` of a level into caller-owned host arrays of nrows+1, nnz and nnz entries
 * (sizes from vk_csr_dims).  Columns are ascending within each row.  Works on host-only hierarchies. */
int vk_export_csr(const vk_hierarchy* h, int level, int which, int32_t* ptr, int32_t* col, double* val);

/* Copies the patch lists of a level (>= 1) into host arrays of npatch+1, nslots and npatch entries:
 * DoFs of patch i are dofs[ptr[i] .. ptr[i+1]), ascending; kind 0 = vertex, 1 = edge, 2 = cell.
 * Patches are ordered vertices, then edges (horizontal, vertical, diagonal), then cells. */
int vk_export_patches(const vk_hierarchy* h, int level, int32_t* ptr, int32_t* dofs, int8_t* kind);

/* Velocity and pressure DoF counts of a level (ndof = n_u + n_p; Case 1 of Sec. 3: continuous P_k
 * velocity, continuous P_{k-1} pressure).  Either pointer may be NULL.  Works on host-only hierarchies. */
int vk_ndof(const vk_hierarchy* h, int level, int64_t* n_u, int64_t* n_p);

/* Coordinates of every DoF of a level in the canonical order: xy (host, 2*ndof doubles, may be NULL)
 * receives (x, y) of the DoF's Lagrange node (equispaced nodes of the structured mesh of Sec. 4);
 * kind (host, ndof bytes, may be NULL) receives 0 / 1 for the x / y velocity component and 2 for
 * pressure.  VK_CELL_BDM: the edge point of each normal-flux DoF (kind 3), the cell centroid for the
 * interior moment DoFs (kind 4), the pressure node (kind 2).  Works on host-only hierarchies. */
int vk_export_dof_coords(const vk_hierarchy* h, int level, double* xy, int8_t* kind);

/* Copies the Dirichlet flags (1 = no-slip velocity DoF) of a level into a host array of ndof bytes. */
int vk_export_dirichlet(const vk_hierarchy* h, int level, uint8_t* flags);

/* Counters of the work a hierarchy issued since the last vk_stats_reset. */
typedef struct vk_stats {
  int64_t launches;        /* CUDA kernels launched on behalf of this hierarchy                     */
  int64_t vcycles;         /* V-cycles started on the finest level                                   */
  int64_t apply_launches;  /* finest-level patch-apply launches bracketed by CUDA events            */
  double apply_ms;         /* their summed event durations (ms), measured on the launching stream   */
  double apply_bytes;      /* algorithmic bytes of one finest-level patch sweep:
                              s*sum(n_i^2) inverse entries (s = 8 FP64 and FP32 pairs, 4 FP32)
                              + 4*sum(n_i) DoF indices + 24*ndof (residual, correction in and out) */
  double apply_flops;      /* 2*sum(n_i^2) flops of one finest-level patch-apply launch             */
  double batch_apply_bytes;/* compulsory bytes of one finest-level tensor-core patch apply of
                              vk_solve_batch: 16-bit inverses as stored + index tables as read +
                              64 per DoF (its 16 FP32 residual values, read once) + 64 per slot
                              (16 FP32 corrections written)                                          */
  double batch_apply_flops;/* 32*sum(n_i^2) flops of that launch (16 right-hand sides)              */
  int64_t spmv_launches;   /* finest-level V-cycle residual SpMV launches bracketed by CUDA events   */
  double spmv_ms;          /* their summed event durations (ms)                                      */
  double spmv_bytes;       /* algorithmic bytes of one finest-level residual r = b - A x (FP64):
                              12*nnz (value, column) + 28*ndof (row index, b, x, r)                 */
  double batch_spmv_bytes; /* the same for the 16-right-hand-side FP32 residual of vk_solve_batch:
                              8*nnz + 4*ndof (row pointer) + 192*ndof (16 x b, x, r)               */
  double setup_factor_ms;  /* setup: summed CUDA-event time of the patch-matrix formation and
                              factorisation launches of every smoothed level (not reset)            */
  double setup_ms;         /* setup: host wall time of vk_setup (not reset)                         */
  int32_t graph_pdl;       /* 1 if the whole-solve graph uses programmatic dependent launch          */
} vk_stats;

/* Zeroes the counters; time_kernels = 1 also brackets every finest-level patch-apply launch and
 * every finest-level V-cycle residual SpMV (of vk_solve and of vk_solve_batch) with CUDA events
 * recorded on the stream that launches it. */
int vk_stats_reset(vk_hierarchy* h, int time_kernels);

/* Reads the counters (waits for the recorded events). */
int vk_stats_read(vk_hierarchy* h, vk_stats* out);

/* ---- group solve: several independent solves advanced together ------------------------------- *
 * A group holds up to `max_members` FGMRES solves (vk_solve semantics), each on its own hierarchy,
 * which may differ in mesh size, number of levels and order k.  vk_group_step advances every active
 * member by one FGMRES iteration, and every stage of it is ONE launch over all active members: the
 * V-cycle's residuals, restrictions and prolongations (SELL products of every member's matrices), the
 * patch solves of Algorithm 1 (uneven patches of every member and order in one launch, each member's
 * own storage layout), the weighted sums with the Chebyshev update (Sec. 3), the coarsest-level solves,
 * and the FGMRES projection, Gram-Schmidt, normalisation and Givens kernels.  Levels are matched from
 * the finest down, so members with fewer levels reach their coarsest solve earlier in the cycle.
 * Members join (vk_group_add) and leave (when they converge, hit maxit or fail) between steps, so a
 * serving loop can batch requests continuously.  Each member's arithmetic is exactly that of
 * vk_solve's host-driven loop (use_graph = 0), in the same order, so its iterations, history and x
 * do not depend on the other members.  A hierarchy can be in at most one group member at a time and
 * must not be used by other calls while it is.  All work is queued on the `stream` of each call. */
typedef struct vk_group vk_group;

int vk_group_create(int max_members, vk_group** out);  /* 1 <= max_members <= 24 */
/* Adds a solve of A x = b on h's finest level (b_dev, x_dev: device, ndof doubles, caller-owned until
 * the member finishes); runs its prologue (projection of b, ||b||, first basis vector) and returns
 * its member id in *member.  A zero right-hand side finishes at once with x = 0. */
int vk_group_add(vk_group* g, vk_hierarchy* h, const double* b_dev, double* x_dev, double rtol, int maxit,
                 void* stream, int* member);
/* One FGMRES iteration of every active member (synchronises the stream once to read the convergence
 * flags); members that finish get x written.  *active (may be NULL) receives the members still active. */
int vk_group_step(vk_group* g, void* stream, int* active);
/* vk_group_add with a host right-hand side (ndof doubles, copied on `stream` into the hierarchy's own
 * device staging buffer before the call returns); the solution stays in the hierarchy's staging
 * buffer until vk_group_result copies it out. */
int vk_group_add_host(vk_group* g, vk_hierarchy* h, const double* b_host, double rtol, int maxit, void* stream,
                      int* member);
/* *active = 1 while the member is being solved, 0 once it has finished (result pending). */
int vk_group_active(const vk_group* g, int member, int* active);
/* Result of a finished member: fills *info (history only if info->history is not NULL, maxit + 1
 * doubles), copies its solution to x_host (ndof doubles; may be NULL) and returns the member's status
 * (VK_OK, VK_ERR_NOT_CONVERGED, VK_ERR_NONFINITE, ...); the member id is free again afterwards.
 * VK_ERR_ARG if the member is unknown or still active. */
int vk_group_result(vk_group* g, int member, double* x_host, vk_solve_info* info);
/* Kernels launched by the group since creation (all members together). */
int vk_group_launches(const vk_group* g, int64_t* launches);
void vk_group_destroy(vk_group* g);

/* ---- solve service (continuous batching on one GPU) ------------------------------------------- *
 * A request is one FGMRES solve (vk_solve semantics) of a problem of its own mesh size and order.
 * Requests are taken in arrival order by `slots` threads that find (or build) a resident hierarchy for
 * each.  Hierarchies stay resident between requests (one pool entry serves one request at a time).
 * Admission is by device footprint (vk_footprint): when memory_budget would be exceeded, idle
 * hierarchies are destroyed least recently used first, and a request waits while the memory it needs
 * is held by running solves; a request larger than the whole budget fails with VK_ERR_NO_MEMORY.
 *   VK_SERVE_GROUP (default): engine threads advance the admitted requests together as members of
 *     group solves (vk_group_*): each FGMRES iteration of all members of a group is one launch per
 *     stage, whatever their sizes and orders, and requests join and leave between iterations
 *     (continuous batching).  There is one group (engine thread and CUDA stream) per size bucket of the
 *     finest level (below 2^16, below 2^19 and from 2^19 DoFs), so small requests share launches with
 *     each other without waiting on the iterations of large ones.  At most slots <= 24 requests are in
 *     flight.
 *   VK_SERVE_STREAMS: each slot solves its request alone (vk_solve_host) on its own CUDA stream, so
 *     the solves overlap on the device but share no launch.
 * Results do not depend on the mix: in both modes each request runs the same deterministic arithmetic
 * on its own hierarchy (group members equal vk_solve's host-driven loop bit for bit). */
#define VK_SERVE_GROUP 0
#define VK_SERVE_STREAMS 1
typedef struct vk_server vk_server;

typedef struct vk_server_config {
  int32_t slots;         /* concurrent solves (1..64)                                             */
  int32_t max_per_key;   /* resident hierarchies per (N_coarse, nlevels, k); requests of a key whose
                            hierarchies are all busy wait for one (0 = slots; default 2)          */
  int32_t device;        /* CUDA device ordinal                                                   */
  size_t memory_budget;  /* device bytes for resident hierarchies; 0 = 60% of free memory         */
  vk_options options;    /* options of every hierarchy the server builds                          */
  int32_t mode;          /* VK_SERVE_GROUP (default) or VK_SERVE_STREAMS                           */
} vk_server_config;

typedef struct vk_request {
  vk_problem problem;    /* mesh hierarchy, order and viscosity of this solve                     */
  const double* b;       /* host right-hand side (ndof doubles), copied by vk_server_submit       */
  double rtol;
  int32_t maxit;
} vk_request;

typedef struct vk_result {
  int32_t status;        /* VK_OK, VK_ERR_NOT_CONVERGED, or the error of the solve / setup        */
  int32_t iterations;
  int32_t converged;
  double res0, true_res; /* as in vk_solve_info                                                   */
  double queue_ms;       /* submission -> start on a slot                                         */
  double setup_ms;       /* hierarchy build time charged to this request (0 when resident)        */
  double solve_ms;       /* vk_solve_host time (copies included)                                  */
  double latency_ms;     /* submission -> result ready on the host                                */
} vk_result;

typedef struct vk_server_stats {
  int64_t submitted, completed, failed, builds, evictions;
  int32_t resident;      /* hierarchies currently resident                                        */
  int32_t queued;        /* requests waiting for a slot                                           */
  size_t bytes_used;     /* device bytes of resident hierarchies                                  */
  size_t memory_budget;
  int64_t group_steps;   /* VK_SERVE_GROUP: FGMRES iterations of the group solve (each one launch per
                            stage over its members)                                              */
  int64_t member_steps;  /* VK_SERVE_GROUP: member iterations in them (member_steps / group_steps is
                            the mean number of requests sharing each launch)                      */
} vk_server_stats;

void vk_default_server_config(vk_server_config* c);   /* 4 slots, 2 per key, device 0, budget 0,
                                                         VK_SERVE_GROUP */
int vk_server_create(const vk_server_config* c, vk_server** out);
/* Queues a request; *ticket identifies it for vk_server_wait. */
int vk_server_submit(vk_server* s, const vk_request* r, uint64_t* ticket);
/* Waits for a request (timeout_ms < 0: forever); copies x (ndof doubles) to x_host if not NULL and
 * fills *res.  Returns VK_ERR_TIMEOUT if the result is not ready in time (the request stays queued). */
int vk_server_wait(vk_server* s, uint64_t ticket, double* x_host, vk_result* res, int timeout_ms);
int vk_server_get_stats(vk_server* s, vk_server_stats* out);
/* Cancels a request that is still queued (not yet taken by a slot): its result becomes available to
 * vk_server_wait at once with status VK_ERR_CANCELLED and no solution.  Returns VK_OK, or VK_ERR_ARG
 * if the ticket is unknown, already running or already finished (a running solve is not interrupted). */
int vk_server_cancel(vk_server* s, uint64_t ticket);
/* Finishes the queued requests, stops the workers and frees every hierarchy. */
void vk_server_destroy(vk_server* s);

/* Right-hand side of the manufactured problem of Sec. 4 (Eq. model_problem: u = (sin(pi x) cos(pi y),
 * -cos(pi x) sin(pi y)), p = 0, f = 2 pi^2 nu u) on the finest level, in the canonical order (b_host:
 * ndof doubles): the load integrated with a collapsed Gauss-Legendre rule of k + 5 points per direction,
 * the velocity's boundary values (their nodal interpolant) lifted, b_F = F_F - K_FB g and b_B = g.
 * VK_CELL_BDM: the load against the Piola-mapped basis; the exact velocity has u . n = 0 on the
 * boundary, so the no-flux entries are zero.  Host computation; works on host-only hierarchies. */
int vk_manufactured_rhs(const vk_hierarchy* h, double* b_host);

/* Discretisation errors of a finest-level solution x_dev (device, ndof doubles) of the manufactured
 * problem, the quantities of the stopping-criterion study of Sec. 4.4: errs[0] = relative H^1 velocity
 * error (||u - u_h||_{H^1} / ||u||_{H^1}; broken, cell by cell, for VK_CELL_BDM), errs[1] = relative
 * L^2 velocity error, errs[2] = absolute
 * L^2 pressure error after removing the pressure's mean (p = 0).  Integrated on the device cell by cell
 * with a collapsed (triangles) or tensor (squares) Gauss-Legendre rule of k + 6 points per direction,
 * summed in a fixed order.  errs is
 * a host array of 3 doubles; the call allocates and frees its tables and synchronises `stream`. */
int vk_errors(vk_hierarchy* h, const double* x_dev, double* errs, void* stream);

/* Measurement helper (no counterpart in the paper: it measures the roofline denominator of the FP64
 * kernels).  FMA throughput of the current device in TFLOP/s (2 flops per FMA): precision 0 = FP64,
 * 1 = FP32.  Runs independent FMA chains on every SM, best of 5 launches timed with CUDA events on
 * `stream` (synchronises it); allocates and frees a small device buffer.  VK_ERR_CUDA on failure. */
int vk_measure_fma_rate(int precision, void* stream, double* tflops);

/* Host-only helper: eigenvalues of the m x m row-major real upper-Hessenberg matrix H (the Arnoldi
 * matrix of the eigenvalue estimate).  Returns VK_ERR_INTERNAL if the QR iteration does not converge. */
int vk_hessenberg_eigenvalues(int m, const double* H, double* re, double* im);

#ifdef __cplusplus
}
#endif

#endif /* VK_H */
