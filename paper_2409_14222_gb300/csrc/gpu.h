// Device-side structures and kernel launchers of the Vanka multigrid library (sm_103a).
// Every launcher returns the number of kernels it launched (0 when there is nothing to do).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

namespace vk {
namespace gpu {

// ---- programmatic dependent launch (inside the whole-solve graph, vk_options.graph_pdl) ----------
// While pdl_enabled() is set on the calling thread (during the capture of the FGMRES graph), the
// solve-path launchers issue their kernels with programmatic stream serialisation: a kernel may be
// launched before its predecessor has fully retired, and every such kernel begins with pdl_wait(),
// which blocks until the predecessor grid has completed and its writes are visible, before touching
// memory (so read-after-write and write-after-read order is unchanged).  Launched the ordinary way,
// pdl_wait() is a no-op.  (Triggering the next launch at the start of each kernel was measured slower:
// the early grids took SM slots from the running one.)
bool pdl_enabled();
void set_pdl(bool on);

template <typename... P, typename... A>
inline void launch(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
  if (!pdl_enabled()) {
    kernel<<<grid, block, smem, s>>>(std::forward<A>(args)...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

// Sliced ELLPACK with C = 32 / tpr rows per slice and tpr threads per row (SELL-C-sigma): rows are
// permuted (sorted by length inside windows of 1024 rows) so the rows of a slice have similar
// lengths; slice widths are padded to a multiple of tpr; entry k of row t of a slice is at
// sptr[slice] + C*k + t, so one warp load of values or columns is 256 / 128 contiguous bytes.
// Padding entries have val = 0 and a valid column.  rowof[C*slice + t] is the original row (-1 past
// the end).  tpr is chosen per matrix so that a launch has enough warps to hide load latency.
struct Sell {
  int nrows = 0, nslices = 0, tpr = 1;
  const int64_t* sptr = nullptr;
  const int* swidth = nullptr;
  const int* col = nullptr;
  const double* val = nullptr;
  const int* rowof = nullptr;
};

struct Csr {
  int nrows = 0;
  const int* ptr = nullptr;
  const int* col = nullptr;
  const double* val = nullptr;
};

// Launch shape of a patch application: split = 0 applies every patch of the level in one launch
// (each warp dispatches on its patch's size); split = 1 launches once per size class (ceil(n/4) in
// 1-4, 5-10, 11-19, 20-32, 33-42), each compiled for that class only.  threads = 128 or 256 per block;
// per_sm = 0 gives one warp per patch, per_sm > 0 a persistent grid of per_sm blocks per SM whose
// warps stride over the patches.  The corrections are bit-identical for every shape.
struct ApplySched {
  int split = 0;
  int threads = 256;
  int per_sm = 0;
};

// Size classes of the patch application by ceil(n/4): 1-4, 5-10, 11-19, 20-32, 33-42 (n <= 168).
constexpr int kApplyClasses = 5;
constexpr int kMaxPatch = 168;

// Patch data of one level.  Patches are processed in "work order" (by packed-tile class, largest
// first); a work item is one warp.  slot_ptr / slot_dofs are in canonical patch order.
struct Patches {
  int npatch = 0;
  int ndof = 0;
  int64_t nslots = 0;
  const int* slot_ptr = nullptr;    // npatch + 1
  const int* slot_dofs = nullptr;   // nslots
  const int* work = nullptr;        // npatch: canonical patch id of work item w
  const int64_t* foff = nullptr;    // npatch: offset (elements) of patch p's packed inverse
  const void* factors = nullptr;    // packed inverses: double (FP64), float (FP32) or float2 (FP32 pair)
  int prec = 0;                     // 0 = FP64, 1 = FP32, 2 = FP32 pair (emulated FP64)
  int sym = 0;                      // 1: symmetric tile layout (sym_packed_size), else warp-packed
  int nb_max = 0;                   // largest packed column-group count ceil(n/4) of the level
  // DoF -> slots (ascending canonical patch order), for the atomic-free sum.  The patch solves write
  // the correction of canonical slot s to delta[slot_pos[s]], so the corrections of DoF i are the
  // contiguous range delta[dof_ptr[i] .. dof_ptr[i+1]) in ascending patch order.
  const int* dof_ptr = nullptr;     // ndof + 1
  const int* slot_pos = nullptr;    // nslots
  const double* weight = nullptr;   // per-DoF weight or nullptr (plain sum)
  ApplySched sched;                 // launch shape used by patch_apply
  int nsm = 152;                    // SMs of the device (persistent grids)
  int cls_lo[kApplyClasses] = {};  // work-list range [cls_lo[c], cls_hi[c]) of size class c
  int cls_hi[kApplyClasses] = {};
};

// ---- sparse / vector kernels (kernels_sparse.cu) -------------------------------------------------
int sell_residual(const Sell& A, const double* b, const double* x, double* y, cudaStream_t s);
// rc = R r with rc = 0 at coarse Dirichlet DoFs; x += P ec  (SELL forms of R and P)
int sell_restrict(const Sell& R, const uint8_t* dir_coarse, const double* r, double* rc, cudaStream_t s);
int sell_prolong_add(const Sell& P, const double* ec, double* x, cudaStream_t s);
// deterministic sums: partial sums over a fixed grid of kReduceBlocks blocks, then one block
constexpr int kReduceBlocks = 256;
int dot_partials(const double* x, const double* y, int n, double* partial, cudaStream_t s);
int finalize_sum(const double* partial, int nparts, double* out, cudaStream_t s);
// x[off..off+len) -= mean of that range (mean from a device scalar: sum / len)
// scratch_sum = sum of x[off .. off+len) (the first two kernels of pressure_project)
int pressure_sum(const double* x, int off, int len, double* scratch_partial, double* scratch_sum, cudaStream_t s);
int pressure_project(double* x, int off, int len, double* scratch_partial, double* scratch_sum,
                      cudaStream_t s);
int fill(double* x, double v, int64_t n, cudaStream_t s);
int copy(double* dst, const double* src, int64_t n, cudaStream_t s);
int nonfinite_check(const double* x, int n, int* flag, cudaStream_t s);
int axpy(double a, const double* x, double* y, int n, cudaStream_t s);   // y += a x
int scale(double a, double* x, int n, cudaStream_t s);                   // x *= a
int divide(double a, double* x, int n, cudaStream_t s);                  // x /= a

// ---- patch kernels (kernels_patch.cu) -------------------------------------------------------------
// Gather every patch matrix from the CSR matrix, invert it by Gauss-Jordan with partial pivoting,
// and store it in the warp-packed layout.  status[0] receives 1 + the first singular patch id.
// Returns -1 (nothing launched) when the level has a patch larger than 128 DoFs.
// (the layout written is P.sym's)
// Matrix-free source of the patch matrices (PCPATCH-style, Sec. 3.1): each patch matrix is assembled
// from the element matrices of every cell containing one of its DoFs, restricted to the patch's DoFs,
// without the global matrix.  Entries are summed over the cells in ascending order, the order of the
// global assembly, so the assembled patch matrix equals the gathered one bit for bit.
struct PatchElems {
  int nloc = 0;                  // element DoFs per cell
  int ncell_lower = 0;           // cells below this index have the lower shape
  const int* cell_dofs = nullptr;    // [cell][nloc] global DoF of each element DoF
  const double* kel = nullptr;       // [2][nloc][nloc] element matrices of the two cell shapes
  const int* cell_ptr = nullptr;     // per patch: range of its cells in `cells`
  const int* cells = nullptr;
};
int patch_factor(const Csr& A, const Patches& P, int prec, void* factors, int* status, cudaStream_t s,
                 const PatchElems* elems = nullptr);
// delta[slot] = (A_i^{-1} r[idx_i]) for every patch (one launch for all patches of a level).  With
// FP32-pair inverses r is first split into r2 (ndof float2) and delta holds FP32 pairs.
int patch_apply(const Patches& P, const double* r, float2* r2, double* delta, cudaStream_t s);
// The same with an explicit launch shape (the autotuner's candidates).
int patch_apply_sched(const Patches& P, const ApplySched& sc, const double* r, float2* r2, double* delta,
                      cudaStream_t s);
// Upper bound of ceil(n/4) of size class c (0..4).
constexpr int kApplyClassHi[kApplyClasses] = {4, 10, 19, 32, 42};
// Sum of the slot corrections into each DoF (+ Dirichlet identity), fused with the Chebyshev update:
//   mode 0: z = M^{-1} r                   (out = z)
//   mode 1: d = z / theta; x = d           (first step, zero initial guess)
//   mode 2: d = z / theta; x += d          (first step, given x)
//   mode 3: d = c1 d + c2 z; x += d        (later steps)
int vanka_scatter(const Patches& P, int ndof, const uint8_t* dir, const double* r, const double* delta,
                   int mode, double theta, double c1, double c2, double* out_z, double* d, double* x,
                   cudaStream_t s);
// Size of the packed inverse of an n x n patch (elements): 32 * ceil(n/8) * ceil(n/4).
inline int64_t packed_size(int n) { return 32LL * ((n + 7) / 8) * ((n + 3) / 4); }
// Symmetric tile layout (FP32 and FP32-pair inverses of levels whose patches have at most kSymMaxN
// DoFs).  A_i is a principal submatrix of the symmetric saddle-point matrix, so A_i^{-1} is symmetric:
// with NT = ceil(n/8) blocks of 8 rows / columns, only the 8 x 8 tiles (I, J) with I <= J are stored,
// row-major over I then J, 64 entries each; lane l = i + 8 j of a warp holds the entries (i, j) and
// (i, j + 4) of a tile at positions 2 l and 2 l + 1 (one 16-byte load per lane for FP32 pairs).  An
// off-diagonal entry stores the mean of the two mirrored entries of the computed inverse.
constexpr int kSymMaxN = 80;
inline int64_t sym_packed_size(int n) {
  const int64_t t = (n + 7) / 8;
  return 32LL * t * (t + 1);
}

// ---- dense coarse solve (kernels_dense.cu) --------------------------------------------------------
// Dense bordered matrix [[A, z], [z^T, 0]] (row-major, (n+1)^2) from the CSR coarsest matrix.
int bordered_from_csr(const Csr& A, int n_u, double* M, cudaStream_t s);
// In-place Gauss-Jordan inverse with partial pivoting of the m x m row-major matrix M.
// perm (m ints), fcol (m doubles), piv (1 int) are scratch; status[0] = 1 on a zero pivot.
int gauss_jordan_inverse(double* M, int m, int* perm, double* fcol, int* piv, int* status, cudaStream_t s);
// x = Minv[0:n, 0:n] b, Minv row stride ld.
int dense_gemv(const double* Minv, int n, int ld, const double* b, double* x, cudaStream_t s);

// ---- FGMRES (kernels_krylov.cu) -------------------------------------------------------------------
// partial[i * kReduceBlocks + blk] = partial dot of V[i] (stride ldv) and w, for i = 0..nvec-1
int multi_dot_partials(const double* V, int64_t ldv, int nvec, const double* w, int n, double* partial,
                        cudaStream_t s);
// out[i] = sum of partial[i*kReduceBlocks ...] for i < nvec (one block per i); acc[i] += the same
// sum when acc is not null
int multi_finalize(const double* partial, int nvec, double* out, double* acc, cudaStream_t s);
// w -= sum_i V[i] h[i]
int multi_axpy(const double* V, int64_t ldv, int nvec, const double* h, double* w, int n, cudaStream_t s);
// v = w / hnorm where hnorm = sqrt(*sq); also writes *hout = hnorm
int normalize(const double* w, const double* sq, double* v, double* hout, int n, cudaStream_t s);
// Givens update of FGMRES column j (single thread); see kernels_krylov.cu.
int givens_update(double* H, int ldh, double* cs, double* sn, double* g, double* hist, int j, double rtol,
                   int* flag, cudaStream_t s);
// ---- device-resident FGMRES (whole solve in one CUDA graph with a WHILE conditional node) ----------
// State read and written by the kernels below; j = completed iterations (the loop index).
struct FgState {
  int j;          // iterations completed
  int flags;      // bit 0: converged, bit 1: non-finite residual estimate
  int maxit;
  int pad;
  double rtol;
  double beta;    // ||b_hat||
  double true_res;
};
// beta = sqrt(*sq); g = (beta, 0, ...); hist[0] = beta; j = 0; sets the loop condition.
int fg_init(const double* sq, FgState* st, double* g, double* hist, int kmax, cudaGraphConditionalHandle cond,
            cudaStream_t s);
int fg_scale(double* v, const FgState* st, int n, double* copy, cudaStream_t s);  // v /= beta; copy = v
// one classical Gram-Schmidt pass against V[0..j]: mode 0 writes H[:, j], mode 1 adds to it
int fg_cgs_pass(const double* V, int64_t ld, const FgState* st, double* w, int n, double* partial, double* H,
                int ldh, double* t2, int kmax, int mode, cudaStream_t s);
// V[j+1] = w / sqrt(*sq), H[j+1][j] = sqrt(*sq)
int fg_normalize(const double* w, const double* sq, double* V, int64_t ld, const FgState* st, double* H, int ldh,
                 int n, double* copy, cudaStream_t s);   // also copy = V[j+1], the next V-cycle input
// z's pressure mean removed and z stored as Z[j] (pressure sum, then one fused kernel)
int fg_project_put(double* z, double* Z, int64_t ld, const FgState* st, int n, int n_u, double* partial,
                   double* sum, cudaStream_t s);
// Givens update of column j, residual history, convergence flags, j += 1, loop condition.
int fg_givens(double* H, int ldh, double* cs, double* sn, double* g, double* hist, FgState* st,
              cudaGraphConditionalHandle cond, cudaStream_t s);
// y = H[0:m,0:m]^{-1} g (back substitution, m = j) and x = Z y
int fg_solution(const double* H, int ldh, const double* g, const double* Z, int64_t ld, const FgState* st,
                double* y, double* x, int n, cudaStream_t s);
int fg_finish(FgState* st, const double* sq, cudaStream_t s);                             // true_res = sqrt(*sq)

// ---- multi-right-hand-side (kernels_batch.cu): 16 right-hand sides interleaved per DoF -----------
// SELL-8 layout of a matrix for the 16-right-hand-side products (slices of 8 rows; entry m of row t
// of slice w at sptr[w] + 8 m + t; rowof[8 w + t] = row, -1 past the end); values as FP32 and FP64.
struct SellB {
  int nrows = 0, nslices = 0;
  const int64_t* sptr = nullptr;
  const int* swidth = nullptr;
  const int* col = nullptr;
  const int* rowof = nullptr;
  const float* valf = nullptr;
  const double* vald = nullptr;
};
// y = b - A x (0), A x (1), b + A x (2), mask ? 0 : A x (3) on [n][16] blocks, values `val` of A
template <typename T>
int mm_sell(const SellB& A, const T* val, int mode, const T* b, const uint8_t* mask, const T* x, T* y,
            cudaStream_t s);
int pack_mma(const Patches& P, const double* inv64, const int64_t* foff16, void* frag, float* ascale, bool half,
             cudaStream_t s);
int patch_apply_mma(const Patches& P, const int64_t* foff16, const void* frag, const float* ascale, bool half,
                    int mt_max, const float* rhs, float* delta, cudaStream_t s);
int scatter_mm(const Patches& P, int ndof, const uint8_t* dir, const float* r, const float* delta, int mode,
               float theta, float c1, float c2, float* zout, float* d, float* x, cudaStream_t s);
int coarse_mm(const float* Minv, int n, int ld, const float* B, float* X, cudaStream_t s);
// FP64 coarse solve of 16 right-hand sides: X[n][16] = Minv[0:n, 0:n] B[n][16]
int coarse_mm64(const double* Minv, int n, int ld, const double* B, double* X, cudaStream_t s);
int to_f32(const double* a, float* b, int64_t n, cudaStream_t s);
int to_f64(const float* a, double* b, int64_t n, cudaStream_t s);
int gather_cols(const double* B, int64_t ld, int nrhs, double* Y, int n, cudaStream_t s);
int scatter_cols(const double* Y, double* X, int64_t ld, int nrhs, int n, cudaStream_t s);
// out[v*16 + r] = sum_rows X_v[row][r] W[row][r] for v < nvec (acc[.] += the same when not null)
int mdot_mm(const double* X, int64_t ldx, int nvec, const double* W, int n, double* partial, double* out,
            double* acc, cudaStream_t s);
// W -= sum_v X_v h_v
int maxpy_mm(const double* X, int64_t ldx, int nvec, const double* h, double* W, int n, cudaStream_t s);
// grid of the batched reductions (partial sums per block, summed in a fixed order)
constexpr int kBatchBlocks = 608;
int project_mm(double* X, int lo, int len, double* partial, double* sum, cudaStream_t s);
int normalize_mm(const double* W, const double* sq, const int* active, double* Y, int n, cudaStream_t s);
int combine_mm(const double* Z, int64_t ldz, const int* m, const double* y, int ldy, double* X, int n,
               cudaStream_t s);
int givens_mm(double* H, int ldh, int64_t hstride, double* cs, double* sn, double* g, double* hist,
              const double* hcol, const double* hnrm, int j, double rtol, int* active, int* iters, int* nonfinite,
              cudaStream_t s);
// Tensor-core (tcgen05) patch solves for 16 right-hand sides (kernels_tc.cu).  Size classes of the
// work list: n <= 40 (3 patches per MMA), n <= 64 (2), n <= 128 (1); each class is cut into groups
// of that many patches.  A group's scaled 16-bit inverses are stored as the exact shared-memory image
// of the MMA's A operand (128 rows = the G patches stacked, 8x8 core matrices), K chunk by K chunk, so
// one bulk copy of 2048 bytes per K chunk of 8 columns moves a whole group.
struct TcClass {
  int ngroups = 0;
  const int* gdof = nullptr;     // [ngroups][G][K] DoF of row k of slot j (-1 past the patch)
  const int* gpos = nullptr;     // [ngroups][128] delta row of accumulator lane t (-1: none)
  const int2* gslot = nullptr;   // [ngroups][G] (n, patch id); n = 0: empty slot
  const int4* gmeta = nullptr;   // [ngroups] (byte offset of the A image: low, high word; bytes; 0)
  const float* gscale = nullptr; // [ngroups][G] the patch's inverse scale, filled by tc_fill_scale
};
struct TcPatches {
  int nsm = 152;
  TcClass cls[3];
  const uint8_t* frag = nullptr;
};
// Patches per group, K (padded patch size) and size cap of class c.
constexpr int kTcG[3] = {3, 2, 1}, kTcK[3] = {48, 64, 128}, kTcCap[3] = {40, 64, 128};
// Bytes of the A image of a group whose largest patch has n DoFs: ceil(n/8) K chunks of 2048 bytes.
inline int64_t tc_group_bytes(int nmax) { return 2048LL * ((nmax + 7) / 8); }
// Pack every group's A image from the FP64 inverses (warp-packed layout), scaled by 1 / ascale[p]
// (ascale from pack_mma); gscale of every slot as well.
int pack_tc(const Patches& P, const TcPatches& T, const double* inv64, const float* ascale, bool half, cudaStream_t s);
// delta[slot][16] = unscaled A_i^{-1} R_i for every patch; *err = VK_ERR_TIMEOUT if a bounded wait
// expired.  One launch per non-empty size class.  skip_group >= 0 (a test of the bounded waits):
// the copy of that group of the first launch is announced but never issued, so its wait expires.
int patch_apply_tc(const TcPatches& T, bool half, const float* rhs, float* delta, int* err, int skip_group,
                   cudaStream_t s);

// 16-bit fragment count (uint4 units) of an n x n patch: (ceil(n/16))^2 tiles of 32 lanes
inline int64_t frag_size(int n) { return 32LL * ((n + 15) / 16) * ((n + 15) / 16); }

// FMA throughput of this device (kernels_probe.cu): best of 5 timed launches of independent FMA
// chains over every SM; FP64 or FP32; TFLOP/s (2 flops per FMA), or < 0 on a CUDA error.  scratch:
// device buffer of at least 8 * 256 * 8 * (SM count) bytes (never written in practice).
double fma_rate_tflops(bool fp64, void* scratch, cudaStream_t s);

// ---- discretisation errors (kernels_fem.cu) --------------------------------------------------------
struct FemErrArgs {
  int N = 0, nb = 0, nq = 0, Q = 0, n_u = 0;
  int quad = 0;                 // 1: the N x N squares (Q_k), 0: the 2 N^2 triangles (P_k)
  int bdm = 0;                  // 1: (BDM_k, dP_{k-1}) on the triangles: Piola-mapped vector basis
  const double* sg = nullptr;   // BDM: [cell][nb] DoF signs
  double h = 0.0;
  const int* cv = nullptr;      // [cell][nb] velocity nodes
  const int* cp = nullptr;      // [cell][nq] pressure nodes
  const double *xi = nullptr, *eta = nullptr, *w = nullptr;                  // [Q] reference rule
  const double *phi = nullptr, *dxi = nullptr, *deta = nullptr;             // [Q][nb] P_k basis
  // (BDM: phi = reference values [Q][nb][2], dxi = reference gradients [Q][nb][2][2])
  const double* psi = nullptr;  // [Q][nq] P_{k-1} basis
  const double* x = nullptr;    // solution (canonical DoF order)
};
// sums[0..6] = e_l2, n_l2, e_h1, n_h1 (gradient parts), int p, int p^2, area; partial: 1024 * 7 doubles
int fem_error_sums(const FemErrArgs& a, double* partial, double* sums, cudaStream_t s);

// ---- group kernels: one launch over the members of a group solve (vk_group_*) -------------------
// Each member is an independent solve on its own hierarchy (its own mesh size, order and matrices).
// A group launch processes the work of every member listed in its by-value argument block; item
// ranges of the members are concatenated (prefix[m] .. prefix[m+1]) and a warp, thread or block finds
// its member by a search over the prefix.  Per element, every group kernel does exactly the
// arithmetic of its single-member counterpart, so a member's results do not depend on the others.
constexpr int kGroupMax = 24;

#ifdef __CUDACC__
// Member of a concatenated range: the largest m with prefix[m] <= i (prefix[0] = 0, count members).
__device__ __forceinline__ int group_member(const int* prefix, int count, int i) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}
#endif

struct GroupSpmvArgs {         // y = op(A) x per member (SELL modes of sell_residual etc.)
  int count = 0;
  int prefix[kGroupMax + 1] = {};   // slices
  Sell A[kGroupMax];
  const double* b[kGroupMax] = {};
  const uint8_t* mask[kGroupMax] = {};
  const double* x[kGroupMax] = {};
  double* y[kGroupMax] = {};
};
// mode 0: y = b - A x, 1: y = A x, 2: y = b + A x, 3: y = mask ? 0 : A x
int group_spmv(int mode, const GroupSpmvArgs& a, cudaStream_t s);

struct GroupPatch {            // one level's patches of one member (the fields patch_apply reads)
  const int* work = nullptr;
  const int* slot_ptr = nullptr;
  const int* slot_dofs = nullptr;
  const int64_t* foff = nullptr;
  const void* factors = nullptr;
  const int* slot_pos = nullptr;
  const int* dof_ptr = nullptr;
  const double* weight = nullptr;
  const uint8_t* dir = nullptr;
  int sym = 0, ndof = 0;
};
struct GroupApplyArgs {        // delta = A_i^{-1} r[idx_i] for every patch of every member
  int count = 0, prec = 0;          // prec: VK_PREC_* shared by the members
  int nb_max = 0;                   // largest ceil(n/4) over the members' patches
  int prefix[kGroupMax + 1] = {};   // patches (work items)
  int dprefix[kGroupMax + 1] = {};  // DoFs (FP32-pair split of the residuals)
  GroupPatch P[kGroupMax];
  const double* r[kGroupMax] = {};
  float2* r2[kGroupMax] = {};       // FP32-pair residual (prec 2)
  double* delta[kGroupMax] = {};
};
int group_patch_apply(const GroupApplyArgs& a, cudaStream_t s);

struct GroupScatterArgs {      // sum of the corrections + Dirichlet identity + Chebyshev update
  int count = 0, prec = 0, mode = 0;
  int prefix[kGroupMax + 1] = {};   // DoFs
  GroupPatch P[kGroupMax];
  const double* r[kGroupMax] = {};
  const double* delta[kGroupMax] = {};
  double theta[kGroupMax] = {}, c1[kGroupMax] = {}, c2[kGroupMax] = {};
  double* z[kGroupMax] = {};
  double* d[kGroupMax] = {};
  double* x[kGroupMax] = {};
};
int group_vanka_scatter(const GroupScatterArgs& a, cudaStream_t s);

struct GroupGemvArgs {         // x = Minv[0:n, 0:n] b per member (coarsest bordered inverse)
  int count = 0;
  int prefix[kGroupMax + 1] = {};   // rows
  const double* Minv[kGroupMax] = {};
  int n[kGroupMax] = {}, ld[kGroupMax] = {};
  const double* b[kGroupMax] = {};
  double* x[kGroupMax] = {};
};
int group_dense_gemv(const GroupGemvArgs& a, cudaStream_t s);

struct GroupVecArgs {          // per-member vectors for the FGMRES kernels below
  int count = 0;
  int n[kGroupMax] = {};
  const double* V[kGroupMax] = {};  // basis (leading dimension ld)
  int64_t ld[kGroupMax] = {};
  int nvec[kGroupMax] = {};         // vectors of V used (j + 1)
  double* w[kGroupMax] = {};
  double* partial[kGroupMax] = {};  // member scratch: kReduceBlocks * (kmax + 1) doubles
  double* out[kGroupMax] = {};      // member results (H column, t2, scalar, ...)
  double* acc[kGroupMax] = {};
  int off[kGroupMax] = {}, len[kGroupMax] = {};   // pressure block (projection)
  int prefix[kGroupMax + 1] = {};   // filled by the launchers: elements or vectors of the members
};
// partial sums of V[i] . w, i < nvec (grid kReduceBlocks x sum of nvec), then out[i] (+ acc[i])
int group_multi_dot(const GroupVecArgs& a, cudaStream_t s);
// w -= sum_i V[i] out[i]
int group_multi_axpy(const GroupVecArgs& a, cudaStream_t s);
// w[off .. off+len) -= its mean (out = scratch scalar)
int group_pressure_project(const GroupVecArgs& a, cudaStream_t s);
// out[0] = w . w (through partial)
int group_norm2(const GroupVecArgs& a, cudaStream_t s);
struct GroupGivensArgs {
  int count = 0;
  double* H[kGroupMax] = {};
  int ldh[kGroupMax] = {};
  double *cs[kGroupMax] = {}, *sn[kGroupMax] = {}, *g[kGroupMax] = {}, *hist[kGroupMax] = {};
  int j[kGroupMax] = {};
  double rtol[kGroupMax] = {};
  int* flag[kGroupMax] = {};
  const double* wsq[kGroupMax] = {};   // ||w||^2 of the new basis vector
  const double* w[kGroupMax] = {};
  double* vnext[kGroupMax] = {};       // V[j + 1] = w / ||w||
  int n[kGroupMax] = {};
  int kmax = 0;
};
// H[j+1][j] = ||w||, V[j+1] = w / ||w|| (all members, one launch), then the rotations of column j
// (one block per member); flag[0] converged, flag[1] non-finite
int group_normalize_givens(const GroupGivensArgs& a, cudaStream_t s);

// x = sum_i Z[i] y[i]
int combine(const double* Z, int64_t ldz, int m, const double* y, double* x, int n, cudaStream_t s);
// y = scale * x
int scale_copy(const double* x, const double* scale_inv_sqrt, double* y, int n, cudaStream_t s);

}  // namespace gpu
}  // namespace vk
