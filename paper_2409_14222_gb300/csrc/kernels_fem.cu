// Discretisation errors of a solution of the manufactured problem (Eq. model_problem, Sec. 4.4):
// relative H^1 and L^2 errors of the velocity and the L^2 error of the pressure after removing its
// mean, integrated cell by cell with a collapsed Gauss-Legendre rule on the reference triangle or a
// tensor Gauss-Legendre rule on the reference square.
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

__global__ void k_errors_final(const double* __restrict__ partial, double* __restrict__ out) {
  if (threadIdx.x >= kFemSums) return;
  double v = 0.0;
  for (int b = 0; b < kFemBlocks; ++b) v += partial[b * kFemSums + threadIdx.x];
  out[threadIdx.x] = v;
}

}  // namespace

int fem_error_sums(const FemErrArgs& a, double* partial, double* sums, cudaStream_t s) {
  k_errors<<<kFemBlocks, kFemThreads, 0, s>>>(a, partial);
  k_errors_final<<<1, 32, 0, s>>>(partial, sums);
  return 2;
}

}  // namespace gpu
}  // namespace vk
