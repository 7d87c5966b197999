// FGMRES building blocks (Sec. 3: right-preconditioned FGMRES with the preconditioned Arnoldi
// vectors kept; Sec. 4: relative residual reduction, zero initial guess).  All reductions use a fixed
// grid and a fixed tree, so results do not depend on scheduling.
#include "gpu.h"

namespace vk {
namespace gpu {

namespace {

constexpr int kT = 256;

template <int T>
__device__ double block_sum(double v) {
  __shared__ double sh[T / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < T / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// grid (kReduceBlocks, nvec): block (b, i) sums V[i][rows of b] * w[rows of b]
__global__ void __launch_bounds__(kT) k_multi_dot(const double* __restrict__ V, int64_t ldv,
                                                  const double* __restrict__ w, int n,
                                                  double* __restrict__ partial) {
  const int i = blockIdx.y;
  const double* v = V + ldv * i;
  double s = 0.0;
  for (int r = blockIdx.x * kT + threadIdx.x; r < n; r += kReduceBlocks * kT) s = fma(v[r], w[r], s);
  s = block_sum<kT>(s);
  if (threadIdx.x == 0) partial[int64_t(i) * kReduceBlocks + blockIdx.x] = s;
}

__global__ void __launch_bounds__(kT) k_multi_finalize(const double* __restrict__ partial,
                                                       double* __restrict__ out, double* __restrict__ acc) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < kReduceBlocks; b += kT) s += partial[int64_t(i) * kReduceBlocks + b];
  s = block_sum<kT>(s);
  if (threadIdx.x == 0) {
    out[i] = s;
    if (acc) acc[i] += s;
  }
}

__global__ void k_multi_axpy(const double* __restrict__ V, int64_t ldv, int nvec, const double* __restrict__ h,
                             double* __restrict__ w, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = 0.0;
  for (int i = 0; i < nvec; ++i) s = fma(V[ldv * i + r], h[i], s);
  w[r] -= s;
}

// may run in place (v == w)
__global__ void k_normalize(const double* w, const double* sq, double* v, double* hout, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const double nrm = sqrt(*sq);
  if (r == 0 && hout) *hout = nrm;
  if (r < n) v[r] = nrm > 0.0 ? w[r] / nrm : w[r];
}

// Apply the previous rotations to column j of H (column-major, leading dimension ldh), build the new
// rotation that zeroes H[j+1][j], update the rotated right-hand side g and the residual history.
// flag[0] = 1 once |g[j+1]| <= rtol * hist[0]; flag[1] = 1 if the estimate is not finite.
__global__ void k_givens(double* __restrict__ H, int ldh, double* __restrict__ cs, double* __restrict__ sn,
                         double* __restrict__ g, double* __restrict__ hist, int j, double rtol, int* flag) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* h = H + int64_t(j) * ldh;
  for (int i = 0; i < j; ++i) {
    const double t = __dadd_rn(__dmul_rn(cs[i], h[i]), __dmul_rn(sn[i], h[i + 1]));
    h[i + 1] = __dadd_rn(__dmul_rn(-sn[i], h[i]), __dmul_rn(cs[i], h[i + 1]));
    h[i] = t;
  }
  const double den = hypot(h[j], h[j + 1]);
  const double c = h[j] / den, s = h[j + 1] / den;
  cs[j] = c;
  sn[j] = s;
  h[j] = den;
  h[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  const double est = fabs(g[j + 1]);
  hist[j + 1] = est;
  flag[0] = est <= rtol * hist[0] ? 1 : 0;
  flag[1] = isfinite(est) ? 0 : 1;
}

// x[r] = sum_i y[i] Z[i][r], summed in increasing i from zero
__global__ void k_combine(const double* __restrict__ Z, int64_t ldz, int m, const double* __restrict__ y,
                          double* __restrict__ x, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = 0.0;
  for (int i = 0; i < m; ++i) s = __dadd_rn(s, __dmul_rn(y[i], Z[ldz * i + r]));
  x[r] = s;
}

__global__ void k_scale_copy(const double* __restrict__ x, const double* __restrict__ sq, double* __restrict__ y,
                             int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double nrm = sqrt(*sq);
  y[r] = x[r] / nrm;
}

}  // namespace

int multi_dot_partials(const double* V, int64_t ldv, int nvec, const double* w, int n, double* partial,
                        cudaStream_t s) {
  if (nvec <= 0) return 0;
  k_multi_dot<<<dim3(kReduceBlocks, nvec), kT, 0, s>>>(V, ldv, w, n, partial);
  return 1;
}

int multi_finalize(const double* partial, int nvec, double* out, double* acc, cudaStream_t s) {
  if (nvec <= 0) return 0;
  k_multi_finalize<<<nvec, kT, 0, s>>>(partial, out, acc);
  return 1;
}

int multi_axpy(const double* V, int64_t ldv, int nvec, const double* h, double* w, int n, cudaStream_t s) {
  k_multi_axpy<<<(n + kT - 1) / kT, kT, 0, s>>>(V, ldv, nvec, h, w, n);
  return 1;
}

int normalize(const double* w, const double* sq, double* v, double* hout, int n, cudaStream_t s) {
  k_normalize<<<(n + kT - 1) / kT, kT, 0, s>>>(w, sq, v, hout, n);
  return 1;
}

int givens_update(double* H, int ldh, double* cs, double* sn, double* g, double* hist, int j, double rtol,
                   int* flag, cudaStream_t s) {
  k_givens<<<1, 32, 0, s>>>(H, ldh, cs, sn, g, hist, j, rtol, flag);
  return 1;
}

int combine(const double* Z, int64_t ldz, int m, const double* y, double* x, int n, cudaStream_t s) {
  k_combine<<<(n + kT - 1) / kT, kT, 0, s>>>(Z, ldz, m, y, x, n);
  return 1;
}

int scale_copy(const double* x, const double* sq, double* y, int n, cudaStream_t s) {
  k_scale_copy<<<(n + kT - 1) / kT, kT, 0, s>>>(x, sq, y, n);
  return 1;
}

}  // namespace gpu
}  // namespace vk
