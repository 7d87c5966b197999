// FMA-rate probe: the denominator of the ALU roofline of the FP64 kernels (the FP64 patch apply, the
// coarse GEMV and the FP64 block products are bound by the FP64 pipe on this part).  Every thread
// runs kChains independent chains a <- a * m + c (one FMA each step), so the pipe never waits on one
// result; the grid covers every SM several times over.  The chains converge to c / (1 - m) = 1 and
// never reach a denormal or an overflow; the results are written behind a condition the compiler
// cannot decide, so no FMA is removed.
#include <algorithm>

#include "gpu.h"

namespace vk {
namespace gpu {

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_chain(int iters, T m, T c, T* out) {
  T a[kChains];
#pragma unroll
  for (int u = 0; u < kChains; ++u) a[u] = T(threadIdx.x + u) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kChains; ++u) a[u] = fma(a[u], m, c);
  }
  T s = T(0);
#pragma unroll
  for (int u = 0; u < kChains; ++u) s += a[u];
  if (s == T(-1)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true; keeps the chains live
}

}  // namespace

double fma_rate_tflops(bool fp64, void* scratch, cudaStream_t s) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1.0;
  // FP64: a few warps per SM already fill the narrow FP64 pipe; FP32 needs every scheduler busy
  const int blocks = nsm * (fp64 ? 4 : 8);
  const int iters = fp64 ? 4096 : 65536;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.0;
  }
  float best = 1e30f;
  for (int rep = 0; rep < 6; ++rep) {   // the first launch is a warm-up
    cudaEventRecord(e0, s);
    if (fp64)
      k_fma_chain<double><<<blocks, kProbeThreads, 0, s>>>(iters, 0.999999, 1e-6, static_cast<double*>(scratch));
    else
      k_fma_chain<float><<<blocks, kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-4f, static_cast<float*>(scratch));
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return -1.0;
  const double fmas = double(blocks) * kProbeThreads * iters * kChains;
  return 2.0 * fmas / (double(best) * 1e-3) / 1e12;
}

}  // namespace gpu
}  // namespace vk
