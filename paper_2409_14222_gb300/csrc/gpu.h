// Device-side structures and kernel launchers of the Vanka multigrid library (sm_103a).
// Every launcher returns the number of kernels it launched (0 when there is nothing to do).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace vk {
namespace gpu {

// Sliced ELLPACK, slice height 32 (SELL-32-sigma): rows are permuted (sorted by length inside windows
// of 1024 rows) so the 32 rows of a slice have similar lengths; within a slice, entry k of lane t is
// at sptr[slice] + 32*k + t, so one warp load of values or columns is 256 / 128 contiguous bytes.
// Padding entries have val = 0 and a valid column.  rowof[pos] is the original row (-1 past the end).
struct Sell {
  int nrows = 0, nslices = 0;
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

// Patch data of one level.  Patches are processed in "work order" (by packed-tile class, largest
// first); a work item is one warp.  slot_ptr / slot_dofs are in canonical patch order.
struct Patches {
  int npatch = 0;
  int64_t nslots = 0;
  const int* slot_ptr = nullptr;    // npatch + 1
  const int* slot_dofs = nullptr;   // nslots
  const int* work = nullptr;        // npatch: canonical patch id of work item w
  const int64_t* foff = nullptr;    // npatch: offset (elements) of patch p's packed inverse
  const void* factors = nullptr;    // packed inverses: double (FP64) or float (FP32)
  int prec = 0;                     // 0 = FP64, 1 = FP32
  int nb_max = 0;                   // largest packed column-group count ceil(n/4) of the level
  // DoF -> slots (ascending canonical patch order), for the atomic-free sum
  const int* dof_ptr = nullptr;     // ndof + 1
  const int* dof_slot = nullptr;    // nslots
  const double* weight = nullptr;   // per-DoF weight or nullptr (plain sum)
};

// ---- sparse / vector kernels (kernels_sparse.cu) -------------------------------------------------
int sell_residual(const Sell& A, const double* b, const double* x, double* y, cudaStream_t s);
int csr_restrict(const Csr& R, const uint8_t* dir_coarse, const double* r, double* rc, cudaStream_t s);
int csr_prolong_add(const Csr& P, const double* ec, double* x, cudaStream_t s);
// deterministic sums: partial sums over a fixed grid of kReduceBlocks blocks, then one block
constexpr int kReduceBlocks = 256;
int dot_partials(const double* x, const double* y, int n, double* partial, cudaStream_t s);
int finalize_sum(const double* partial, int nparts, double* out, cudaStream_t s);
// x[off..off+len) -= mean of that range (mean from a device scalar: sum / len)
int pressure_project(double* x, int off, int len, double* scratch_partial, double* scratch_sum,
                      cudaStream_t s);
int fill(double* x, double v, int64_t n, cudaStream_t s);
int copy(double* dst, const double* src, int64_t n, cudaStream_t s);
int nonfinite_check(const double* x, int n, int* flag, cudaStream_t s);
int axpy(double a, const double* x, double* y, int n, cudaStream_t s);   // y += a x
int scale(double a, double* x, int n, cudaStream_t s);                   // x *= a

// ---- patch kernels (kernels_patch.cu) -------------------------------------------------------------
// Gather every patch matrix from the CSR matrix, invert it by Gauss-Jordan with partial pivoting,
// and store it in the warp-packed layout.  status[0] receives 1 + the first singular patch id.
int patch_factor(const Csr& A, const Patches& P, int prec, void* factors, int* status, cudaStream_t s);
// delta[slot] = (A_i^{-1} r[idx_i]) for every patch (one launch for all patches of a level).
int patch_apply(const Patches& P, const double* r, double* delta, cudaStream_t s);
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
// x = sum_i Z[i] y[i]
int combine(const double* Z, int64_t ldz, int m, const double* y, double* x, int n, cudaStream_t s);
// y = scale * x
int scale_copy(const double* x, const double* scale_inv_sqrt, double* y, int n, cudaStream_t s);

}  // namespace gpu
}  // namespace vk
