// Discretisation errors of a solution of the manufactured problem (Eq. model_problem, Sec. 4.4):
// relative H^1 and L^2 errors of the velocity and the L^2 error of the pressure after removing its
// mean, integrated cell by cell with a collapsed Gauss-Legendre rule on the reference triangle or a
// tensor Gauss-Legendre rule on the reference square; for (BDM_k, dP_{k-1}) the broken H^1 error, cell
// by cell, of the Piola-mapped velocity.
// One thread per cell over a fixed grid, fixed reduction tree: the sums do not depend on scheduling.
#include "gpu.h"

namespace vk {
namespace gpu {

namespace {

constexpr int kFemThreads = 128;
constexpr int kFemBlocks = 1024;
constexpr int kFemSums = 7;   // e_l2, n_l2, e_h1 (gradient part), n_h1 (gradient part), p_int, p_sq, area

__global__ void __launch_bounds__(kFemThreads) k_errors(FemErrArgs a, double* __restrict__ partial) {
  double acc[kFemSums];
#pragma unroll
  for (int i = 0; i < kFemSums; ++i) acc[i] = 0.0;
  const int ncell = (a.quad ? 1 : 2) * a.N * a.N;
  const double pi = 3.14159265358979323846;
  for (int c = blockIdx.x * kFemThreads + threadIdx.x; c < ncell; c += kFemBlocks * kFemThreads) {
    // vertex v0 and edge vectors of the cell (units of h): lower (i,j),(i+1,j),(i,j+1);
    // upper (i+1,j),(i+1,j+1),(i,j+1)
    // squares: cell (i, j) = j N + i, x = h (i + xi), y = h (j + eta)
    const int q = c % (a.N * a.N), i = q % a.N, j = q / a.N;
    const bool up = !a.quad && c >= a.N * a.N;
    const double x0 = a.h * (up ? i + 1 : i), y0 = a.h * j;
    const double J00 = up ? 0.0 : a.h, J01 = up ? -a.h : 0.0, J10 = up ? a.h : 0.0, J11 = a.h;
    const double det = J00 * J11 - J01 * J10, adet = fabs(det);
    const double T00 = J11 / det, T01 = -J10 / det, T10 = -J01 / det, T11 = J00 / det;
    const int* vn = a.cv + int64_t(c) * a.nb;
    const int* pn = a.cp + int64_t(c) * a.nq;
    for (int t = 0; t < a.Q; ++t) {
      const double X = x0 + J00 * a.xi[t] + J01 * a.eta[t], Y = y0 + J10 * a.xi[t] + J11 * a.eta[t];
      const double w = a.w[t] * adet;
      double u1 = 0.0, u2 = 0.0, g11 = 0.0, g12 = 0.0, g21 = 0.0, g22 = 0.0, ph = 0.0;
      for (int b = 0; b < a.nb; ++b) {
        const double f = a.phi[t * a.nb + b];
        const double gx = T00 * a.dxi[t * a.nb + b] + T01 * a.deta[t * a.nb + b];
        const double gy = T10 * a.dxi[t * a.nb + b] + T11 * a.deta[t * a.nb + b];
        const double x1 = a.x[2 * vn[b]], x2 = a.x[2 * vn[b] + 1];
        u1 += f * x1;
        u2 += f * x2;
        g11 += gx * x1;
        g12 += gy * x1;
        g21 += gx * x2;
        g22 += gy * x2;
      }
      for (int p = 0; p < a.nq; ++p) ph += a.psi[t * a.nq + p] * a.x[a.n_u + pn[p]];
      const double sx = sin(pi * X), cx = cos(pi * X), sy = sin(pi * Y), cy = cos(pi * Y);
      const double e1 = sx * cy, e2 = -cx * sy;
      const double E11 = pi * cx * cy, E12 = -pi * sx * sy, E21 = pi * sx * sy, E22 = -pi * cx * cy;
      acc[0] += w * ((u1 - e1) * (u1 - e1) + (u2 - e2) * (u2 - e2));
      acc[1] += w * (e1 * e1 + e2 * e2);
      acc[2] += w * ((g11 - E11) * (g11 - E11) + (g12 - E12) * (g12 - E12) + (g21 - E21) * (g21 - E21) +
                     (g22 - E22) * (g22 - E22));
      acc[3] += w * (E11 * E11 + E12 * E12 + E21 * E21 + E22 * E22);
      acc[4] += w * ph;
      acc[5] += w * ph * ph;
      acc[6] += w;
    }
  }
  __shared__ double sh[kFemThreads / 32][kFemSums];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kFemSums; ++i) {
    double v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < kFemSums) {
    double v = 0.0;
    for (int w = 0; w < kFemThreads / 32; ++w) v += sh[w][threadIdx.x];
    partial[blockIdx.x * kFemSums + threadIdx.x] = v;
  }
}

// (BDM_k, dP_{k-1}): the velocity of cell c is sum_i s_i x_i J vhat_i / det J (contravariant Piola map,
// s_i the cell's DoF signs), its gradient sum_i s_i x_i J (grad vhat_i) J^{-1} / det J.
__device__ __forceinline__ void bdm_point(const FemErrArgs& a, int c, int t, const double J[2][2], double det,
                                          const double Ji[2][2], double u[2], double g[2][2]) {
  u[0] = u[1] = 0.0;
  g[0][0] = g[0][1] = g[1][0] = g[1][1] = 0.0;
  double rv[2] = {0.0, 0.0}, rg[2][2] = {{0.0, 0.0}, {0.0, 0.0}};   // reference-cell sums
  for (int b = 0; b < a.nb; ++b) {
    const double cf = a.sg[int64_t(c) * a.nb + b] * a.x[a.cv[int64_t(c) * a.nb + b]];
    const double* v = a.phi + (int64_t(t) * a.nb + b) * 2;
    const double* d = a.dxi + (int64_t(t) * a.nb + b) * 4;
    rv[0] += cf * v[0];
    rv[1] += cf * v[1];
    rg[0][0] += cf * d[0];
    rg[0][1] += cf * d[1];
    rg[1][0] += cf * d[2];
    rg[1][1] += cf * d[3];
  }
  for (int i = 0; i < 2; ++i) {
    u[i] = (J[i][0] * rv[0] + J[i][1] * rv[1]) / det;
    for (int j = 0; j < 2; ++j) {
      double s = 0.0;
      for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) s += J[i][p] * rg[p][q] * Ji[q][j];
      g[i][j] = s / det;
    }
  }
}

__global__ void __launch_bounds__(kFemThreads) k_errors_bdm(FemErrArgs a, double* __restrict__ partial) {
  double acc[kFemSums];
#pragma unroll
  for (int i = 0; i < kFemSums; ++i) acc[i] = 0.0;
  const int ncell = 2 * a.N * a.N;
  const double pi = 3.14159265358979323846;
  for (int c = blockIdx.x * kFemThreads + threadIdx.x; c < ncell; c += kFemBlocks * kFemThreads) {
    const int q = c % (a.N * a.N), i = q % a.N, j = q / a.N;
    const bool up = c >= a.N * a.N;
    const double x0 = a.h * (up ? i + 1 : i), y0 = a.h * j;
    const double J[2][2] = {{up ? 0.0 : a.h, up ? -a.h : 0.0}, {up ? a.h : 0.0, a.h}};
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0], adet = fabs(det);
    const double Ji[2][2] = {{J[1][1] / det, -J[0][1] / det}, {-J[1][0] / det, J[0][0] / det}};
    for (int t = 0; t < a.Q; ++t) {
      const double X = x0 + J[0][0] * a.xi[t] + J[0][1] * a.eta[t], Y = y0 + J[1][0] * a.xi[t] + J[1][1] * a.eta[t];
      const double w = a.w[t] * adet;
      double u[2], g[2][2];
      bdm_point(a, c, t, J, det, Ji, u, g);
      double ph = 0.0;
      for (int p = 0; p < a.nq; ++p) ph += a.psi[t * a.nq + p] * a.x[a.n_u + a.cp[int64_t(c) * a.nq + p]];
      const double sx = sin(pi * X), cx = cos(pi * X), sy = sin(pi * Y), cy = cos(pi * Y);
      const double e[2] = {sx * cy, -cx * sy};
      const double E[2][2] = {{pi * cx * cy, -pi * sx * sy}, {pi * sx * sy, -pi * cx * cy}};
      for (int m = 0; m < 2; ++m) {
        acc[0] += w * (u[m] - e[m]) * (u[m] - e[m]);
        acc[1] += w * e[m] * e[m];
        for (int n = 0; n < 2; ++n) {
          acc[2] += w * (g[m][n] - E[m][n]) * (g[m][n] - E[m][n]);
          acc[3] += w * E[m][n] * E[m][n];
        }
      }
      acc[4] += w * ph;
      acc[5] += w * ph * ph;
      acc[6] += w;
    }
  }
  __shared__ double sh[kFemThreads / 32][kFemSums];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kFemSums; ++i) {
    double v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < kFemSums) {
    double v = 0.0;
    for (int w = 0; w < kFemThreads / 32; ++w) v += sh[w][threadIdx.x];
    partial[blockIdx.x * kFemSums + threadIdx.x] = v;
  }
}

__global__ void k_errors_final(const double* __restrict__ partial, double* __restrict__ out) {
  if (threadIdx.x >= kFemSums) return;
  double v = 0.0;
  for (int b = 0; b < kFemBlocks; ++b) v += partial[b * kFemSums + threadIdx.x];
  out[threadIdx.x] = v;
}

}  // namespace

int fem_error_sums(const FemErrArgs& a, double* partial, double* sums, cudaStream_t s) {
  if (a.bdm)
    k_errors_bdm<<<kFemBlocks, kFemThreads, 0, s>>>(a, partial);
  else
    k_errors<<<kFemBlocks, kFemThreads, 0, s>>>(a, partial);
  k_errors_final<<<1, 32, 0, s>>>(partial, sums);
  return 2;
}

}  // namespace gpu
}  // namespace vk
