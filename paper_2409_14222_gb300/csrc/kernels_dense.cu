// Coarsest-level solve: the bordered system [[A_0, z], [z^T, 0]] with z = (0_u, 1_p) (the constant
// pressure, kernel of the Dirichlet system, Sec. 2) is inverted once at setup by Gauss-Jordan
// elimination with partial pivoting, and each V-cycle applies the top-left block of the inverse as a
// dense GEMV (the paper does not name its coarse solver; a direct solve is read).
#include "gpu.h"

namespace vk {
namespace gpu {

namespace {

__global__ void k_bordered(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                           const double* __restrict__ val, int n_u, double* __restrict__ M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int ld = n + 1;
  if (i >= n) return;
  for (int e = ptr[i]; e < ptr[i + 1]; ++e) M[int64_t(i) * ld + col[e]] = val[e];
  const double zi = i >= n_u ? 1.0 : 0.0;
  M[int64_t(i) * ld + n] = zi;
  M[int64_t(n) * ld + i] = zi;
}

__global__ void k_zero(double* M, int64_t len) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < len) M[i] = 0.0;
}

// Pivot search of column k (first maximal |M[i][k]|, i >= k) and the saved column for the
// elimination in post-interchange order: fcol[i] = M[i][k] for i != k, piv; fcol[piv] = M[k][k].
__global__ void __launch_bounds__(1024) k_gj_pivot(double* __restrict__ M, int m, int k, int* __restrict__ perm,
                                                   double* __restrict__ fcol, int* __restrict__ piv,
                                                   double* __restrict__ pivval, int* status) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int spiv;
  const int tid = threadIdx.x;
  double best = -1.0;
  int bi = m;
  for (int i = k + tid; i < m; i += 1024) {
    const double v = fabs(M[int64_t(i) * m + k]);
    if (v > best) { best = v; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
  }
  if ((tid & 31) == 0) { sv[tid >> 5] = best; si[tid >> 5] = bi; }
  __syncthreads();
  if (tid == 0) {
    double bv = sv[0];
    int bidx = si[0];
    for (int w = 1; w < 32; ++w)
      if (sv[w] > bv || (sv[w] == bv && si[w] < bidx)) { bv = sv[w]; bidx = si[w]; }
    if (!(bv > 0.0) || !isfinite(bv)) {
      *status = 1;
      bidx = k;
    }
    spiv = bidx;
    *piv = bidx;
    perm[k] = bidx;
    *pivval = M[int64_t(bidx) * m + k];
  }
  __syncthreads();
  const int p = spiv;
  for (int i = tid; i < m; i += 1024) {
    if (i == k) continue;
    fcol[i] = (i == p) ? M[int64_t(k) * m + k] : M[int64_t(i) * m + k];
  }
}

// Interchange rows k and piv and scale the new row k (its diagonal becomes 1 / pivot).
__global__ void k_gj_swap_scale(double* __restrict__ M, int m, int k, const int* __restrict__ piv,
                                const double* __restrict__ pivval) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int p = *piv;
  const double pv = *pivval;
  const double a = M[int64_t(k) * m + j], b = M[int64_t(p) * m + j];
  if (p != k) M[int64_t(p) * m + j] = a;
  M[int64_t(k) * m + j] = (j == k ? 1.0 : (p != k ? b : a)) / pv;
}

__global__ void k_gj_eliminate(double* __restrict__ M, int m, int k, const double* __restrict__ fcol) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= m || i == k) return;
  const int64_t idx = int64_t(i) * m + j;
  M[idx] = (j == k ? 0.0 : M[idx]) - fcol[i] * M[int64_t(k) * m + j];
}

__global__ void k_gj_unscramble(double* __restrict__ M, int m, const int* __restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double* row = M + int64_t(i) * m;
  for (int k = m - 1; k >= 0; --k) {
    const int q = perm[k];
    if (q != k) {
      const double t = row[k];
      row[k] = row[q];
      row[q] = t;
    }
  }
}

// x[row] = Minv[row][0:n] . b: one block of 128 threads per row (enough warps per SM for the FP64
// pipe and the loads), two partial sums per thread, fixed combination order.
__device__ __forceinline__ void gemv_row(int row, const double* __restrict__ Minv, int n, int ld,
                                         const double* __restrict__ b, double* __restrict__ x) {
  __shared__ double sh[4];
  const int tid = threadIdx.x, lane = tid & 31;
  const double* a = Minv + int64_t(row) * ld;
  double s0 = 0.0, s1 = 0.0;
  int j = tid;
  for (; j + 128 < n; j += 256) {
    s0 = fma(__ldg(a + j), __ldg(b + j), s0);
    s1 = fma(__ldg(a + j + 128), __ldg(b + j + 128), s1);
  }
  if (j < n) s0 = fma(__ldg(a + j), __ldg(b + j), s0);
  double s = s0 + s1;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) sh[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) x[row] = (sh[0] + sh[1]) + (sh[2] + sh[3]);
}

__global__ void __launch_bounds__(128) k_dense_gemv(const double* __restrict__ Minv, int n, int ld,
                                                    const double* __restrict__ b, double* __restrict__ x) {
  pdl_wait();
  gemv_row(blockIdx.x, Minv, n, ld, b, x);
}

__global__ void __launch_bounds__(128) k_group_gemv(const __grid_constant__ GroupGemvArgs a) {
  const int gr = blockIdx.x;
  const int m = group_member(a.prefix, a.count, gr);
  gemv_row(gr - a.prefix[m], a.Minv[m], a.n[m], a.ld[m], a.b[m], a.x[m]);
}

}  // namespace

int bordered_from_csr(const Csr& A, int n_u, double* M, cudaStream_t s) {
  const int n = A.nrows;
  const int64_t len = int64_t(n + 1) * (n + 1);
  k_zero<<<int((len + 255) / 256), 256, 0, s>>>(M, len);
  k_bordered<<<(n + 255) / 256, 256, 0, s>>>(n, A.ptr, A.col, A.val, n_u, M);
  return 2;
}

int gauss_jordan_inverse(double* M, int m, int* perm, double* fcol, int* piv, int* status, cudaStream_t s) {
  // pivval lives right after the m-entry fcol scratch
  double* pivval = fcol + m;
  const int tb = 256;
  for (int k = 0; k < m; ++k) {
    k_gj_pivot<<<1, 1024, 0, s>>>(M, m, k, perm, fcol, piv, pivval, status);
    k_gj_swap_scale<<<(m + tb - 1) / tb, tb, 0, s>>>(M, m, k, piv, pivval);
    k_gj_eliminate<<<dim3((m + tb - 1) / tb, m), tb, 0, s>>>(M, m, k, fcol);
  }
  k_gj_unscramble<<<(m + 127) / 128, 128, 0, s>>>(M, m, perm);
  return 3 * m + 1;
}

int group_dense_gemv(const GroupGemvArgs& a, cudaStream_t s) {
  if (a.count == 0 || a.prefix[a.count] == 0) return 0;
  k_group_gemv<<<a.prefix[a.count], 128, 0, s>>>(a);
  return 1;
}

int dense_gemv(const double* Minv, int n, int ld, const double* b, double* x, cudaStream_t s) {
  launch(k_dense_gemv, dim3(n), dim3(128), 0, s, Minv, n, ld, b, x);
  return 1;
}

}  // namespace gpu
}  // namespace vk
