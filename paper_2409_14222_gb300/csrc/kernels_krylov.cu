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

// Rotations of FGMRES column j (column-major H, leading dimension ldh): apply the previous rotations,
// build the one that zeroes H[j+1][j], update g and the history.  The column and the rotations are
// first loaded into shared memory by all threads; one thread then runs the sequential recurrence.
// Returns (in thread 0) the new estimate |g[j+1]|.
__device__ double givens_column(double* __restrict__ H, int ldh, double* __restrict__ cs, double* __restrict__ sn,
                                double* __restrict__ g, double* __restrict__ hist, int j) {
  extern __shared__ double sh[];
  double* h = sh;                 // j + 2
  double* c = sh + (j + 2);       // j
  double* sv = c + j;             // j
  double* col = H + int64_t(j) * ldh;
  for (int i = threadIdx.x; i < j + 2; i += blockDim.x) h[i] = col[i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    c[i] = cs[i];
    sv[i] = sn[i];
  }
  __syncthreads();
  double est = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < j; ++i) {
      const double t = __dadd_rn(__dmul_rn(c[i], h[i]), __dmul_rn(sv[i], h[i + 1]));
      h[i + 1] = __dadd_rn(__dmul_rn(-sv[i], h[i]), __dmul_rn(c[i], h[i + 1]));
      h[i] = t;
    }
    const double den = hypot(h[j], h[j + 1]);
    const double cj = h[j] / den, sj = h[j + 1] / den;
    cs[j] = cj;
    sn[j] = sj;
    h[j] = den;
    h[j + 1] = 0.0;
    g[j + 1] = -sj * g[j];
    g[j] = cj * g[j];
    est = fabs(g[j + 1]);
    hist[j + 1] = est;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < j + 2; i += blockDim.x) col[i] = h[i];
  return est;
}

// flag[0] = 1 once |g[j+1]| <= rtol * hist[0]; flag[1] = 1 if the estimate is not finite.
__global__ void k_givens(double* __restrict__ H, int ldh, double* __restrict__ cs, double* __restrict__ sn,
                         double* __restrict__ g, double* __restrict__ hist, int j, double rtol, int* flag) {
  const double est = givens_column(H, ldh, cs, sn, g, hist, j);
  if (threadIdx.x == 0) {
    flag[0] = est <= rtol * hist[0] ? 1 : 0;
    flag[1] = isfinite(est) ? 0 : 1;
  }
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

// may run in place (y == x)
__global__ void k_scale_copy(const double* x, const double* __restrict__ sq, double* y, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double nrm = sqrt(*sq);
  y[r] = x[r] / nrm;
}

// ---------------- device-resident FGMRES kernels (iteration index read from FgState) -------------
__global__ void k_fg_init(const double* __restrict__ sq, FgState* st, double* __restrict__ g,
                          double* __restrict__ hist, int kmax, cudaGraphConditionalHandle cond) {
  pdl_wait();
  const double beta = sqrt(*sq);
  for (int i = threadIdx.x; i <= kmax; i += blockDim.x) g[i] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int flags = 0;
    if (!isfinite(beta)) flags |= 2;
    else if (beta == 0.0) flags |= 1;
    st->beta = beta;
    st->j = 0;
    st->flags = flags;
    st->true_res = 0.0;
    g[0] = beta;
    hist[0] = beta;
    cudaGraphSetConditional(cond, (flags == 0 && st->maxit > 0) ? 1u : 0u);
  }
}

// v /= beta, and the same values into copy (the V-cycle input of the first iteration)
__global__ void k_fg_scale(double* v, const FgState* __restrict__ st, int n, double* __restrict__ copy) {
  pdl_wait();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double beta = st->beta;
  double x = v[r];
  if (beta > 0.0 && isfinite(beta)) {
    x = x / beta;
    v[r] = x;
  }
  copy[r] = x;
}

// Grid (kReduceBlocks, ceil(kmax / kFgVB)): block (b, g) forms the partial dots of rows
// {b*kT + t + k*kReduceBlocks*kT} (the partition of k_multi_dot) with the basis vectors
// g*kFgVB .. g*kFgVB + kFgVB - 1 that are <= j (w read once for the group); blocks of groups beyond j
// return at once.  Each vector's partial is summed in the same element order and combined by the same
// tree as block_sum, so the values equal those of k_multi_dot.
constexpr int kFgVB = 8;
__global__ void __launch_bounds__(kT) k_fg_mdot(const double* __restrict__ V, int64_t ld,
                                                const FgState* __restrict__ st, const double* __restrict__ w,
                                                int n, double* __restrict__ partial) {
  pdl_wait();
  __shared__ double sh[kFgVB][kT / 32];
  const int j = st->j, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  {
    const int i0 = blockIdx.y * kFgVB;
    if (i0 > j) return;
    double s[kFgVB];
#pragma unroll
    for (int u = 0; u < kFgVB; ++u) s[u] = 0.0;
    for (int r = blockIdx.x * kT + threadIdx.x; r < n; r += kReduceBlocks * kT) {
      const double wr = w[r];
#pragma unroll
      for (int u = 0; u < kFgVB; ++u)
        if (i0 + u <= j) s[u] = fma(V[ld * (i0 + u) + r], wr, s[u]);
    }
#pragma unroll
    for (int u = 0; u < kFgVB; ++u) {
      for (int o = 16; o > 0; o >>= 1) s[u] += __shfl_xor_sync(0xffffffffu, s[u], o);
      if (lane == 0) sh[u][warp] = s[u];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int u = 0; u < kFgVB; ++u) {
        double v = lane < kT / 32 ? sh[u][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && i0 + u <= j) partial[int64_t(i0 + u) * kReduceBlocks + blockIdx.x] = v;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kT) k_fg_mfin(const double* __restrict__ partial, const FgState* __restrict__ st,
                                                double* __restrict__ H, int ldh, double* __restrict__ t2, int mode) {
  pdl_wait();
  const int i = blockIdx.x, j = st->j;
  if (i > j) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < kReduceBlocks; b += kT) s += partial[int64_t(i) * kReduceBlocks + b];
  s = block_sum<kT>(s);
  if (threadIdx.x == 0) {
    double* col = H + int64_t(j) * ldh;
    if (mode == 0) {
      col[i] = s;
    } else {
      t2[i] = s;
      col[i] += s;
    }
  }
}

__global__ void k_fg_maxpy(const double* __restrict__ V, int64_t ld, const FgState* __restrict__ st,
                           const double* __restrict__ H, int ldh, const double* __restrict__ t2, int mode,
                           double* __restrict__ w, int n) {
  pdl_wait();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int j = st->j;
  const double* h = mode == 0 ? H + int64_t(j) * ldh : t2;
  double s = 0.0;
#pragma unroll 4
  for (int i = 0; i <= j; ++i) s = fma(V[ld * i + r], h[i], s);
  w[r] -= s;
}

__global__ void k_fg_normalize(const double* __restrict__ w, const double* __restrict__ sq, double* __restrict__ V,
                               int64_t ld, const FgState* __restrict__ st, double* __restrict__ H, int ldh, int n,
                               double* __restrict__ copy) {
  pdl_wait();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = st->j;
  const double nrm = sqrt(*sq);
  if (r == 0) H[int64_t(j) * ldh + j + 1] = nrm;
  if (r < n) {
    const double x = nrm > 0.0 ? w[r] / nrm : w[r];
    V[ld * (j + 1) + r] = x;
    copy[r] = x;   // the next iteration's V-cycle input
  }
}

// The pressure part of z loses its mean (the same arithmetic as the projection's subtraction), and z
// is stored as column j of Z.
__global__ void k_fg_project_put(double* __restrict__ z, double* __restrict__ Z, int64_t ld,
                                 const FgState* __restrict__ st, int n, int n_u, const double* __restrict__ sum) {
  pdl_wait();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double x = z[r];
  if (r >= n_u) {
    x -= *sum / double(n - n_u);
    z[r] = x;
  }
  Z[ld * st->j + r] = x;
}

__global__ void k_fg_givens(double* __restrict__ H, int ldh, double* __restrict__ cs, double* __restrict__ sn,
                            double* __restrict__ g, double* __restrict__ hist, FgState* st,
                            cudaGraphConditionalHandle cond) {
  pdl_wait();
  const int j = st->j;
  const double est = givens_column(H, ldh, cs, sn, g, hist, j);
  if (threadIdx.x == 0) {
    int flags = 0;
    if (!isfinite(est)) flags |= 2;
    else if (est <= st->rtol * hist[0]) flags |= 1;
    st->flags = flags;
    st->j = j + 1;
    cudaGraphSetConditional(cond, (flags == 0 && j + 1 < st->maxit) ? 1u : 0u);
  }
}

// Back substitution with one warp: y[i] = (g[i] - sum_{k>i} H[i][k] y[k]) / H[i][i].
__global__ void k_fg_backsolve(const double* __restrict__ H, int ldh, const double* __restrict__ g,
                               const FgState* __restrict__ st, double* __restrict__ y) {
  pdl_wait();
  extern __shared__ double ys[];
  const int m = st->j, lane = threadIdx.x;
  for (int i = m - 1; i >= 0; --i) {
    double s = 0.0;
    for (int k = i + 1 + lane; k < m; k += 32) s = fma(H[int64_t(k) * ldh + i], ys[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) ys[i] = (g[i] - s) / H[int64_t(i) * ldh + i];
    __syncwarp();
  }
  for (int i = lane; i < m; i += 32) y[i] = ys[i];
}

__global__ void k_fg_combine(const double* __restrict__ Z, int64_t ldz, const FgState* __restrict__ st,
                             const double* __restrict__ y, double* __restrict__ x, int n) {
  pdl_wait();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int m = st->j;
  double s = 0.0;
  for (int i = 0; i < m; ++i) s = __dadd_rn(s, __dmul_rn(y[i], Z[ldz * i + r]));
  x[r] = s;
}

__global__ void k_fg_finish(FgState* st, const double* __restrict__ sq) {
  pdl_wait();
  st->true_res = sqrt(*sq);
}

// ---- group forms: the same partitions, orders and trees as the single-solve kernels ------------
// block (b, v) of the grid: member m and basis vector i of the concatenated vector list
__global__ void __launch_bounds__(kT) k_group_multi_dot(const __grid_constant__ GroupVecArgs a) {
  const int gv = blockIdx.y;
  const int m = group_member(a.prefix, a.count, gv), i = gv - a.prefix[m];
  const double* v = a.V[m] + a.ld[m] * i;
  const double* w = a.w[m];
  const int n = a.n[m];
  double s = 0.0;
  for (int r = blockIdx.x * kT + threadIdx.x; r < n; r += kReduceBlocks * kT) s = fma(v[r], w[r], s);
  s = block_sum<kT>(s);
  if (threadIdx.x == 0) a.partial[m][int64_t(i) * kReduceBlocks + blockIdx.x] = s;
}

__global__ void __launch_bounds__(kT) k_group_multi_finalize(const __grid_constant__ GroupVecArgs a) {
  const int gv = blockIdx.x;
  const int m = group_member(a.prefix, a.count, gv), i = gv - a.prefix[m];
  double s = 0.0;
  for (int b = threadIdx.x; b < kReduceBlocks; b += kT) s += a.partial[m][int64_t(i) * kReduceBlocks + b];
  s = block_sum<kT>(s);
  if (threadIdx.x == 0) {
    a.out[m][i] = s;
    if (a.acc[m]) a.acc[m][i] += s;
  }
}

__global__ void k_group_multi_axpy(const __grid_constant__ GroupVecArgs a) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= a.prefix[a.count]) return;
  const int m = group_member(a.prefix, a.count, gi), r = gi - a.prefix[m];
  const double* V = a.V[m];
  const double* h = a.out[m];
  const int64_t ld = a.ld[m];
  double s = 0.0;
  for (int i = 0; i < a.nvec[m]; ++i) s = fma(V[ld * i + r], h[i], s);
  a.w[m][r] -= s;
}

// mode 0: partial sums of w[off .. off+len) (k_sum_partials); mode 1: of w . w over n (k_dot_partials)
template <int kMode>
__global__ void __launch_bounds__(kT) k_group_sum(const __grid_constant__ GroupVecArgs a) {
  const int m = blockIdx.y;
  double s = 0.0;
  if (kMode == 0) {
    const double* x = a.w[m] + a.off[m];
    for (int i = blockIdx.x * kT + threadIdx.x; i < a.len[m]; i += kReduceBlocks * kT) s += x[i];
  } else {
    const double* x = a.w[m];
    for (int i = blockIdx.x * kT + threadIdx.x; i < a.n[m]; i += kReduceBlocks * kT) s = fma(x[i], x[i], s);
  }
  s = block_sum<kT>(s);
  if (threadIdx.x == 0) a.partial[a.count > 0 ? m : 0][blockIdx.x] = s;
}

__global__ void __launch_bounds__(kT) k_group_finalize(const __grid_constant__ GroupVecArgs a) {
  const int m = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < kReduceBlocks; i += kT) s += a.partial[m][i];
  s = block_sum<kT>(s);
  if (threadIdx.x == 0) a.out[m][0] = s;
}

__global__ void k_group_subtract_mean(const __grid_constant__ GroupVecArgs a) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= a.prefix[a.count]) return;
  const int m = group_member(a.prefix, a.count, gi), i = gi - a.prefix[m];
  double* x = a.w[m] + a.off[m];
  x[i] -= *a.out[m] / double(a.len[m]);
}

__global__ void k_group_normalize(const __grid_constant__ GroupGivensArgs a, const __grid_constant__ GroupVecArgs pre) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= pre.prefix[pre.count]) return;
  const int m = group_member(pre.prefix, pre.count, gi), r = gi - pre.prefix[m];
  const double nrm = sqrt(*a.wsq[m]);
  if (r == 0) a.H[m][int64_t(a.j[m]) * a.ldh[m] + a.j[m] + 1] = nrm;
  a.vnext[m][r] = nrm > 0.0 ? a.w[m][r] / nrm : a.w[m][r];
}

// one block per member: the rotations of column j (givens_column) and the convergence flags
__global__ void k_group_givens(const __grid_constant__ GroupGivensArgs a) {
  const int m = blockIdx.x;
  const int j = a.j[m];
  const double est = givens_column(a.H[m], a.ldh[m], a.cs[m], a.sn[m], a.g[m], a.hist[m], j);
  if (threadIdx.x == 0) {
    a.flag[m][0] = est <= a.rtol[m] * a.hist[m][0] ? 1 : 0;
    a.flag[m][1] = isfinite(est) ? 0 : 1;
  }
}

}  // namespace

int group_multi_dot(const GroupVecArgs& a0, cudaStream_t s) {
  if (a0.count == 0) return 0;
  GroupVecArgs a = a0;
  a.prefix[0] = 0;
  for (int m = 0; m < a.count; ++m) a.prefix[m + 1] = a.prefix[m] + a.nvec[m];
  if (a.prefix[a.count] == 0) return 0;
  k_group_multi_dot<<<dim3(kReduceBlocks, a.prefix[a.count]), kT, 0, s>>>(a);
  k_group_multi_finalize<<<a.prefix[a.count], kT, 0, s>>>(a);
  return 2;
}

int group_multi_axpy(const GroupVecArgs& a0, cudaStream_t s) {
  if (a0.count == 0) return 0;
  GroupVecArgs a = a0;
  a.prefix[0] = 0;
  for (int m = 0; m < a.count; ++m) a.prefix[m + 1] = a.prefix[m] + a.n[m];
  k_group_multi_axpy<<<(a.prefix[a.count] + kT - 1) / kT, kT, 0, s>>>(a);
  return 1;
}

int group_pressure_project(const GroupVecArgs& a0, cudaStream_t s) {
  if (a0.count == 0) return 0;
  GroupVecArgs a = a0;
  a.prefix[0] = 0;
  for (int m = 0; m < a.count; ++m) a.prefix[m + 1] = a.prefix[m] + a.len[m];
  k_group_sum<0><<<dim3(kReduceBlocks, a.count), kT, 0, s>>>(a);
  k_group_finalize<<<a.count, kT, 0, s>>>(a);
  k_group_subtract_mean<<<(a.prefix[a.count] + kT - 1) / kT, kT, 0, s>>>(a);
  return 3;
}

int group_norm2(const GroupVecArgs& a, cudaStream_t s) {
  if (a.count == 0) return 0;
  k_group_sum<1><<<dim3(kReduceBlocks, a.count), kT, 0, s>>>(a);
  k_group_finalize<<<a.count, kT, 0, s>>>(a);
  return 2;
}

int group_normalize_givens(const GroupGivensArgs& a, cudaStream_t s) {
  if (a.count == 0) return 0;
  GroupVecArgs pre;
  pre.count = a.count;
  pre.prefix[0] = 0;
  for (int m = 0; m < a.count; ++m) pre.prefix[m + 1] = pre.prefix[m] + a.n[m];
  k_group_normalize<<<(pre.prefix[a.count] + kT - 1) / kT, kT, 0, s>>>(a, pre);
  // shared memory of the largest column: 3 * kmax + 2 doubles
  k_group_givens<<<a.count, 128, (3 * (a.kmax + 1) + 2) * sizeof(double), s>>>(a);
  return 2;
}

int fg_init(const double* sq, FgState* st, double* g, double* hist, int kmax, cudaGraphConditionalHandle cond,
            cudaStream_t s) {
  launch(k_fg_init, dim3(1), dim3(kT), 0, s, sq, st, g, hist, kmax, cond);
  return 1;
}

int fg_scale(double* v, const FgState* st, int n, double* copy, cudaStream_t s) {
  launch(k_fg_scale, dim3((n + kT - 1) / kT), dim3(kT), 0, s, v, st, n, copy);
  return 1;
}

int fg_project_put(double* z, double* Z, int64_t ld, const FgState* st, int n, int n_u, double* partial,
                   double* sum, cudaStream_t s) {
  int k = pressure_sum(z, n_u, n - n_u, partial, sum, s);
  launch(k_fg_project_put, dim3((n + kT - 1) / kT), dim3(kT), 0, s, z, Z, ld, st, n, n_u, sum);
  return k + 1;
}

int fg_cgs_pass(const double* V, int64_t ld, const FgState* st, double* w, int n, double* partial, double* H,
                int ldh, double* t2, int kmax, int mode, cudaStream_t s) {
  launch(k_fg_mdot, dim3(dim3(kReduceBlocks, (kmax + kFgVB - 1) / kFgVB)), dim3(kT), 0, s, V, ld, st, w, n, partial);
  launch(k_fg_mfin, dim3(kmax), dim3(kT), 0, s, partial, st, H, ldh, t2, mode);
  launch(k_fg_maxpy, dim3((n + kT - 1) / kT), dim3(kT), 0, s, V, ld, st, H, ldh, t2, mode, w, n);
  return 3;
}

int fg_normalize(const double* w, const double* sq, double* V, int64_t ld, const FgState* st, double* H, int ldh,
                 int n, double* copy, cudaStream_t s) {
  launch(k_fg_normalize, dim3((n + kT - 1) / kT), dim3(kT), 0, s, w, sq, V, ld, st, H, ldh, n, copy);
  return 1;
}

int fg_givens(double* H, int ldh, double* cs, double* sn, double* g, double* hist, FgState* st,
              cudaGraphConditionalHandle cond, cudaStream_t s) {
  // shared memory for the largest column: 3 * kmax + 2 doubles (ldh = kmax + 1)
  launch(k_fg_givens, dim3(1), dim3(128), (3 * ldh + 2) * sizeof(double), s, H, ldh, cs, sn, g, hist, st, cond);
  return 1;
}

int fg_solution(const double* H, int ldh, const double* g, const double* Z, int64_t ld, const FgState* st,
                double* y, double* x, int n, cudaStream_t s) {
  launch(k_fg_backsolve, dim3(1), dim3(32), ldh * sizeof(double), s, H, ldh, g, st, y);
  launch(k_fg_combine, dim3((n + kT - 1) / kT), dim3(kT), 0, s, Z, ld, st, y, x, n);
  return 2;
}

int fg_finish(FgState* st, const double* sq, cudaStream_t s) {
  launch(k_fg_finish, dim3(1), dim3(1), 0, s, st, sq);
  return 1;
}

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
  k_givens<<<1, 128, (3 * j + 2) * sizeof(double), s>>>(H, ldh, cs, sn, g, hist, j, rtol, flag);
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
