// Sparse and vector kernels: SELL-32 SpMV / residual, CSR restriction and prolongation, and
// deterministic (fixed-order) reductions.  FP64 throughout.
//
// Residual r = b - A x of every relaxed level and the FGMRES product w = A z (Sec. 3, Algorithm 1's
// local right-hand sides); R = P^T restriction and P prolongation (Sec. 3, grid transfers).
#include "gpu.h"

namespace vk {
namespace gpu {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n, int t = kThreads) { return int((n + t - 1) / t); }

// SELL-C with T = 32 / C threads per row: warp w owns slice w (C rows); lane l = t + C q works on row
// t of the slice and on the entries k = T m + q of that row.  Entry k of row t is stored at
// sptr[w] + C k + t, so for each m the warp reads the 32 consecutive entries sptr[w] + 32 m + l.
// Loads are issued 8 steps ahead of the FMAs (the kernel is latency-bound otherwise); the T partial
// sums of a row are combined by a fixed xor tree.
//   kMode 0: y = b - A x          1: y = A x
//   kMode 2: y = b + A x          3: y = mask ? 0 : A x   (mask = Dirichlet flags of the output)
// (b and y may be the same vector: each row reads b[row] before writing y[row].)
template <int kMode, int T>
__device__ __forceinline__ void sell_slice(int warp, int lane, const int64_t* __restrict__ sptr,
                                           const int* __restrict__ sw, const int* __restrict__ col,
                                           const double* __restrict__ val, const int* __restrict__ rowof,
                                           const double* b, const uint8_t* __restrict__ mask,
                                           const double* __restrict__ x, double* y) {
  constexpr int C = 32 / T;
  const int t = lane % C;
  const int row = rowof[warp * C + t];
  const int steps = sw[warp] / T;
  const int64_t base = sptr[warp] + lane;
  const int* cp = col + base;
  const double* vp = val + base;
  double sum = 0.0;
  int m = 0;
  constexpr int U = 8;
  for (; m + U <= steps; m += U) {
    int c[U];
    double v[U], xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = __ldg(cp + 32 * (m + u));
      v[u] = __ldg(vp + 32 * (m + u));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = x[c[u]];
#pragma unroll
    for (int u = 0; u < U; ++u) sum = fma(v[u], xv[u], sum);
  }
  for (; m < steps; ++m) sum = fma(__ldg(vp + 32 * m), x[__ldg(cp + 32 * m)], sum);
#pragma unroll
  for (int o = C; o < 32; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane >= C || row < 0) return;
  if (kMode == 0) y[row] = b[row] - sum;
  if (kMode == 1) y[row] = sum;
  if (kMode == 2) y[row] = b[row] + sum;
  if (kMode == 3) y[row] = mask[row] ? 0.0 : sum;
}

template <int kMode, int T>
__global__ void __launch_bounds__(kThreads) k_sell(int nslices, const int64_t* __restrict__ sptr,
                                                   const int* __restrict__ sw, const int* __restrict__ col,
                                                   const double* __restrict__ val, const int* __restrict__ rowof,
                                                   const double* b, const uint8_t* __restrict__ mask,
                                                   const double* __restrict__ x, double* y) {
  pdl_wait();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= nslices) return;
  sell_slice<kMode, T>(warp, threadIdx.x & 31, sptr, sw, col, val, rowof, b, mask, x, y);
}

// One warp per slice of any member's matrix; the member's own threads-per-row layout.
template <int kMode>
__global__ void __launch_bounds__(kThreads) k_group_sell(const __grid_constant__ GroupSpmvArgs a) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= a.prefix[a.count]) return;
  const int m = group_member(a.prefix, a.count, gw);
  const Sell& A = a.A[m];
  const int w = gw - a.prefix[m], lane = threadIdx.x & 31;
  switch (A.tpr) {
    case 1: sell_slice<kMode, 1>(w, lane, A.sptr, A.swidth, A.col, A.val, A.rowof, a.b[m], a.mask[m], a.x[m], a.y[m]); break;
    case 2: sell_slice<kMode, 2>(w, lane, A.sptr, A.swidth, A.col, A.val, A.rowof, a.b[m], a.mask[m], a.x[m], a.y[m]); break;
    case 4: sell_slice<kMode, 4>(w, lane, A.sptr, A.swidth, A.col, A.val, A.rowof, a.b[m], a.mask[m], a.x[m], a.y[m]); break;
    default: sell_slice<kMode, 8>(w, lane, A.sptr, A.swidth, A.col, A.val, A.rowof, a.b[m], a.mask[m], a.x[m], a.y[m]); break;
  }
}

template <int kMode>
int launch_sell(const Sell& A, const double* b, const uint8_t* mask, const double* x, double* y, cudaStream_t s) {
  if (A.nslices == 0) return 0;
  const int g = blocks_for(int64_t(A.nslices) * 32);
  switch (A.tpr) {
    case 1:
      launch(k_sell<kMode, 1>, dim3(g), dim3(kThreads), 0, s, A.nslices, A.sptr, A.swidth, A.col, A.val, A.rowof, b, mask, x, y);
      break;
    case 2:
      launch(k_sell<kMode, 2>, dim3(g), dim3(kThreads), 0, s, A.nslices, A.sptr, A.swidth, A.col, A.val, A.rowof, b, mask, x, y);
      break;
    case 4:
      launch(k_sell<kMode, 4>, dim3(g), dim3(kThreads), 0, s, A.nslices, A.sptr, A.swidth, A.col, A.val, A.rowof, b, mask, x, y);
      break;
    default:
      launch(k_sell<kMode, 8>, dim3(g), dim3(kThreads), 0, s, A.nslices, A.sptr, A.swidth, A.col, A.val, A.rowof, b, mask, x, y);
      break;
  }
  return 1;
}

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
  return v;  // valid in thread 0
}

__global__ void __launch_bounds__(kThreads) k_dot_partials(const double* __restrict__ x,
                                                           const double* __restrict__ y, int n,
                                                           double* __restrict__ partial) {
  pdl_wait();
  double s = 0.0;
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += kReduceBlocks * kThreads)
    s = fma(x[i], y[i], s);
  s = block_sum<kThreads>(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_sum_partials(const double* __restrict__ x, int n,
                                                           double* __restrict__ partial) {
  pdl_wait();
  double s = 0.0;
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += kReduceBlocks * kThreads) s += x[i];
  s = block_sum<kThreads>(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_finalize(const double* __restrict__ partial, int nparts,
                                                       double* __restrict__ out) {
  pdl_wait();
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kThreads) s += partial[i];
  s = block_sum<kThreads>(s);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_subtract_mean(double* __restrict__ x, int len, const double* __restrict__ sum) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  x[i] -= *sum / double(len);
}

__global__ void k_fill(double* x, double v, int64_t n) {
  pdl_wait();
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) x[i] = v;
}

__global__ void k_copy(double* __restrict__ d, const double* __restrict__ s, int64_t n) {
  pdl_wait();
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) d[i] = s[i];
}

__global__ void k_nonfinite(const double* __restrict__ x, int n, int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(x[i])) *flag = 1;
}

__global__ void k_axpy(double a, const double* __restrict__ x, double* __restrict__ y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __dsub_rn(y[i], __dmul_rn(-a, x[i]));  // y - (-a) x, unfused
}

__global__ void k_scale(double a, double* __restrict__ x, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = x[i] * a;
}

__global__ void k_divide(double a, double* __restrict__ x, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = x[i] / a;
}

}  // namespace

namespace {
thread_local bool t_pdl = false;
}

bool pdl_enabled() { return t_pdl; }
void set_pdl(bool on) { t_pdl = on; }

int divide(double a, double* x, int n, cudaStream_t s) {
  if (n <= 0) return 0;
  k_divide<<<blocks_for(n), kThreads, 0, s>>>(a, x, n);
  return 1;
}

int axpy(double a, const double* x, double* y, int n, cudaStream_t s) {
  if (n <= 0) return 0;
  k_axpy<<<blocks_for(n), kThreads, 0, s>>>(a, x, y, n);
  return 1;
}

int scale(double a, double* x, int n, cudaStream_t s) {
  if (n <= 0) return 0;
  k_scale<<<blocks_for(n), kThreads, 0, s>>>(a, x, n);
  return 1;
}

int group_spmv(int mode, const GroupSpmvArgs& a, cudaStream_t s) {
  if (a.count == 0 || a.prefix[a.count] == 0) return 0;
  const int g = blocks_for(int64_t(a.prefix[a.count]) * 32);
  switch (mode) {
    case 0: k_group_sell<0><<<g, kThreads, 0, s>>>(a); break;
    case 1: k_group_sell<1><<<g, kThreads, 0, s>>>(a); break;
    case 2: k_group_sell<2><<<g, kThreads, 0, s>>>(a); break;
    default: k_group_sell<3><<<g, kThreads, 0, s>>>(a); break;
  }
  return 1;
}

int sell_residual(const Sell& A, const double* b, const double* x, double* y, cudaStream_t s) {
  return b ? launch_sell<0>(A, b, nullptr, x, y, s) : launch_sell<1>(A, nullptr, nullptr, x, y, s);
}

int sell_restrict(const Sell& R, const uint8_t* dir_coarse, const double* r, double* rc, cudaStream_t s) {
  return launch_sell<3>(R, nullptr, dir_coarse, r, rc, s);
}

int sell_prolong_add(const Sell& P, const double* ec, double* x, cudaStream_t s) {
  return launch_sell<2>(P, x, nullptr, ec, x, s);
}



int dot_partials(const double* x, const double* y, int n, double* partial, cudaStream_t s) {
  launch(k_dot_partials, dim3(kReduceBlocks), dim3(kThreads), 0, s, x, y, n, partial);
  return 1;
}

int finalize_sum(const double* partial, int nparts, double* out, cudaStream_t s) {
  launch(k_finalize, dim3(1), dim3(kThreads), 0, s, partial, nparts, out);
  return 1;
}

int pressure_sum(const double* x, int off, int len, double* scratch_partial, double* scratch_sum, cudaStream_t s) {
  if (len <= 0) return 0;
  launch(k_sum_partials, dim3(kReduceBlocks), dim3(kThreads), 0, s, x + off, len, scratch_partial);
  launch(k_finalize, dim3(1), dim3(kThreads), 0, s, scratch_partial, kReduceBlocks, scratch_sum);
  return 2;
}

int pressure_project(double* x, int off, int len, double* scratch_partial, double* scratch_sum,
                      cudaStream_t s) {
  if (len <= 0) return 0;
  launch(k_sum_partials, dim3(kReduceBlocks), dim3(kThreads), 0, s, x + off, len, scratch_partial);
  launch(k_finalize, dim3(1), dim3(kThreads), 0, s, scratch_partial, kReduceBlocks, scratch_sum);
  launch(k_subtract_mean, dim3(blocks_for(len)), dim3(kThreads), 0, s, x + off, len, scratch_sum);
  return 3;
}

int fill(double* x, double v, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  launch(k_fill, dim3(blocks_for(n)), dim3(kThreads), 0, s, x, v, n);
  return 1;
}

int copy(double* dst, const double* src, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  launch(k_copy, dim3(blocks_for(n)), dim3(kThreads), 0, s, dst, src, n);
  return 1;
}

int nonfinite_check(const double* x, int n, int* flag, cudaStream_t s) {
  if (n <= 0) return 0;
  k_nonfinite<<<blocks_for(n), kThreads, 0, s>>>(x, n, flag);
  return 1;
}

}  // namespace gpu
}  // namespace vk
