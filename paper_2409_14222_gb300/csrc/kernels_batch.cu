// Multi-right-hand-side kernels (vk_solve_batch): block vectors hold kNR = 16 right-hand sides
// interleaved per DoF ([ndof][16], the 16 values of a DoF are contiguous), so a matrix entry is read
// once for 16 products and a gathered row is one 64-byte (FP32) or 128-byte (FP64) access.
//
// The V-cycle preconditioner runs in FP32 (FP32 matrices, FP32 block vectors); the patch solves of
// Algorithm 1 become a dense contraction delta_i[n x 16] = A_i^{-1}[n x n] R_i[n x 16] per patch,
// done on the tensor cores with 16-bit inputs (BF16 or FP16) and FP32 accumulation: mma.sync
// m16n8k16.  A_i^{-1} is stored scaled by its largest magnitude, pre-packed in the A-fragment order
// of the instruction (one 16-byte load per lane per 16x16 tile); each right-hand-side column of R_i
// is scaled by its own largest magnitude, so a column's result does not depend on the other columns.
// The outer FGMRES (residual w = A z, orthogonalisation, Givens) stays in FP64.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "gpu.h"

namespace vk {
namespace gpu {

namespace {

constexpr int kNR = 16;
constexpr int kT = 256;

inline int nblk(int64_t n, int t = kT) { return int((n + t - 1) / t); }

template <int T>
__device__ double block_sum_d(double v) {
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

// ---- block SpMM, CSR, half-warp per row, lane = right-hand side ---------------------------------
//   kMode 0: y = b - A x   1: y = A x   2: y = b + A x   3: y = mask ? 0 : A x
template <typename T, int kMode>
__global__ void __launch_bounds__(kT) k_mm(int nrows, const int* __restrict__ ptr, const int* __restrict__ col,
                                           const T* __restrict__ val, const T* b, const uint8_t* __restrict__ mask,
                                           const T* __restrict__ x, T* y) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const int r = threadIdx.x & 15;
  if (row >= nrows) return;
  const int e0 = ptr[row], e1 = ptr[row + 1];
  T acc = T(0);
  int e = e0;
  for (; e + 4 <= e1; e += 4) {
    const int c0 = __ldg(col + e), c1 = __ldg(col + e + 1), c2 = __ldg(col + e + 2), c3 = __ldg(col + e + 3);
    const T v0 = __ldg(val + e), v1 = __ldg(val + e + 1), v2 = __ldg(val + e + 2), v3 = __ldg(val + e + 3);
    const T x0 = x[int64_t(c0) * kNR + r], x1 = x[int64_t(c1) * kNR + r];
    const T x2 = x[int64_t(c2) * kNR + r], x3 = x[int64_t(c3) * kNR + r];
    acc = fma(v0, x0, acc);
    acc = fma(v1, x1, acc);
    acc = fma(v2, x2, acc);
    acc = fma(v3, x3, acc);
  }
  for (; e < e1; ++e) acc = fma(__ldg(val + e), x[int64_t(__ldg(col + e)) * kNR + r], acc);
  const int64_t o = int64_t(row) * kNR + r;
  if (kMode == 0) y[o] = b[o] - acc;
  if (kMode == 1) y[o] = acc;
  if (kMode == 2) y[o] = b[o] + acc;
  if (kMode == 3) y[o] = mask[row] ? T(0) : acc;
}

// ---- tensor-core patch apply --------------------------------------------------------------------
template <bool kHalf>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if constexpr (kHalf) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
}

template <bool kHalf>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1) {
  if constexpr (kHalf)
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
  else
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// One warp, one patch of size n <= 16 * MT.  Fragment conventions of mma.m16n8k16 (g = lane >> 2,
// t = lane & 3):  A regs {A[g][2t..2t+1], A[g+8][2t..], A[g][2t+8..], A[g+8][2t+8..]};
// B regs {B[2t..2t+1][g], B[2t+8..2t+9][g]};  D {D[g][2t..2t+1], D[g+8][2t..2t+1]}.
// The N dimension (16 right-hand sides) is two 8-wide tiles.
template <int MT, bool kHalf>
__device__ __forceinline__ void mma_patch(int n, int s0, const int* __restrict__ dofs, const uint4* __restrict__ frag,
                                          float ascale, const float* __restrict__ rhs, const int* __restrict__ pos,
                                          float* __restrict__ delta, int lane) {
  const int g = lane >> 2, t = lane & 3;
  // gather the residual block in B-fragment order: rows k of tile kt, column nt*8 + g
  float rv[MT][2][4];
  float cmax[2] = {0.f, 0.f};
#pragma unroll
  for (int kt = 0; kt < MT; ++kt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = kt * 16 + 2 * t + (q & 1) + (q >> 1) * 8;
        const float v = k < n ? rhs[int64_t(__ldg(dofs + k)) * kNR + nt * 8 + g] : 0.f;
        rv[kt][nt][q] = v;
        cmax[nt] = fmaxf(cmax[nt], fabsf(v));
      }
  // per-column scale: lanes 4g .. 4g+3 hold the rows of column nt*8 + g
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
    cmax[nt] = fmaxf(cmax[nt], __shfl_xor_sync(0xffffffffu, cmax[nt], 1));
    cmax[nt] = fmaxf(cmax[nt], __shfl_xor_sync(0xffffffffu, cmax[nt], 2));
  }
  const float cinv[2] = {cmax[0] > 0.f ? 1.f / cmax[0] : 0.f, cmax[1] > 0.f ? 1.f / cmax[1] : 0.f};
  uint32_t bf[MT][2][2];
#pragma unroll
  for (int kt = 0; kt < MT; ++kt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      bf[kt][nt][0] = pack2<kHalf>(rv[kt][nt][0] * cinv[nt], rv[kt][nt][1] * cinv[nt]);
      bf[kt][nt][1] = pack2<kHalf>(rv[kt][nt][2] * cinv[nt], rv[kt][nt][3] * cinv[nt]);
    }
  // output columns of this lane are 2t, 2t+1 of each n-tile: their scales live in lanes 4*(2t), 4*(2t+1)
  float oscale[2][2];
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
    oscale[nt][0] = ascale * __shfl_sync(0xffffffffu, cmax[nt], 8 * t);
    oscale[nt][1] = ascale * __shfl_sync(0xffffffffu, cmax[nt], 8 * t + 4);
  }
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
    float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < MT; ++kt) {
      const uint4 a = __ldg(frag + (mt * MT + kt) * 32 + lane);
      mma16816<kHalf>(d0, a, bf[kt][0][0], bf[kt][0][1]);
      mma16816<kHalf>(d1, a, bf[kt][1][0], bf[kt][1][1]);
    }
    const int r0 = mt * 16 + g, r1 = r0 + 8;
    if (r0 < n) {
      float* o = delta + int64_t(__ldg(pos + s0 + r0)) * kNR;
      *reinterpret_cast<float2*>(o + 2 * t) = make_float2(d0[0] * oscale[0][0], d0[1] * oscale[0][1]);
      *reinterpret_cast<float2*>(o + 8 + 2 * t) = make_float2(d1[0] * oscale[1][0], d1[1] * oscale[1][1]);
    }
    if (r1 < n) {
      float* o = delta + int64_t(__ldg(pos + s0 + r1)) * kNR;
      *reinterpret_cast<float2*>(o + 2 * t) = make_float2(d0[2] * oscale[0][0], d0[3] * oscale[0][1]);
      *reinterpret_cast<float2*>(o + 8 + 2 * t) = make_float2(d1[2] * oscale[1][0], d1[3] * oscale[1][1]);
    }
  }
}

template <int MT, int MTMAX, bool kHalf>
__device__ __forceinline__ void mma_dispatch(int mt, int n, int s0, const int* dofs, const uint4* frag, float ascale,
                                             const float* rhs, const int* pos, float* delta, int lane) {
  if constexpr (MT <= MTMAX) {
    if (mt == MT)
      mma_patch<MT, kHalf>(n, s0, dofs, frag, ascale, rhs, pos, delta, lane);
    else
      mma_dispatch<MT + 1, MTMAX, kHalf>(mt, n, s0, dofs, frag, ascale, rhs, pos, delta, lane);
  }
}

template <int MTMAX, bool kHalf>
__global__ void __launch_bounds__(kT) k_patch_mma(int npatch, const int* __restrict__ work,
                                                  const int* __restrict__ slot_ptr, const int* __restrict__ slot_dofs,
                                                  const int64_t* __restrict__ foff, const uint4* __restrict__ frag,
                                                  const float* __restrict__ ascale, const float* __restrict__ rhs,
                                                  const int* __restrict__ pos, float* __restrict__ delta) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= npatch) return;
  const int p = work[w];
  const int s0 = slot_ptr[p], n = slot_ptr[p + 1] - s0;
  mma_dispatch<1, MTMAX, kHalf>((n + 15) >> 4, n, s0, slot_dofs + s0, frag + foff[p], ascale[p], rhs, pos, delta,
                                lane);
}

// Pack one patch's FP64 inverse (warp-packed layout of kernels_patch.cu) into scaled 16-bit
// A fragments.  One block per patch.
template <bool kHalf>
__global__ void k_pack_mma(const int* __restrict__ slot_ptr, const int64_t* __restrict__ foff64,
                           const double* __restrict__ inv64, const int64_t* __restrict__ foff16,
                           uint4* __restrict__ frag, float* __restrict__ ascale) {
  const int p = blockIdx.x;
  const int n = slot_ptr[p + 1] - slot_ptr[p];
  const int NB = (n + 3) / 4, NA = (n + 7) / 8, MT = (n + 15) / 16;
  const double* src = inv64 + foff64[p];
  auto at = [&](int row, int col) -> double {
    if (row >= n || col >= n) return 0.0;
    const int a = row >> 3, rr = row & 7, b = col >> 2, cc = col & 3;
    return src[(a * NB + b) * 32 + rr + 8 * cc];
  };
  __shared__ float smax[32];
  float m = 0.f;
  for (int e = threadIdx.x; e < 32 * NA * NB; e += blockDim.x) m = fmaxf(m, float(fabs(src[e])));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = 0.f;
    for (int i = 0; i < int(blockDim.x + 31) / 32; ++i) mm = fmaxf(mm, smax[i]);
    smax[0] = mm > 0.f ? mm : 1.f;
    ascale[p] = smax[0];
  }
  __syncthreads();
  const double inv = 1.0 / double(smax[0]);
  uint4* dst = frag + foff16[p];
  for (int e = threadIdx.x; e < MT * MT * 32; e += blockDim.x) {
    const int tile = e >> 5, lane = e & 31, mt = tile / MT, kt = tile % MT;
    const int g = lane >> 2, t = lane & 3;
    const int r0 = mt * 16 + g, r1 = r0 + 8, c0 = kt * 16 + 2 * t, c1 = c0 + 8;
    uint4 v;
    v.x = pack2<kHalf>(float(at(r0, c0) * inv), float(at(r0, c0 + 1) * inv));
    v.y = pack2<kHalf>(float(at(r1, c0) * inv), float(at(r1, c0 + 1) * inv));
    v.z = pack2<kHalf>(float(at(r0, c1) * inv), float(at(r0, c1 + 1) * inv));
    v.w = pack2<kHalf>(float(at(r1, c1) * inv), float(at(r1, c1 + 1) * inv));
    dst[e] = v;
  }
}

// ---- Vanka sum + Chebyshev update on FP32 block vectors (thread per DoF and right-hand side) ------
__global__ void __launch_bounds__(kT) k_scatter_mm(int ndof, const int* __restrict__ dptr,
                                                   const uint8_t* __restrict__ dir, const float* __restrict__ r,
                                                   const float* __restrict__ delta, int mode, float theta, float c1,
                                                   float c2, float* __restrict__ zout, float* __restrict__ d,
                                                   float* __restrict__ x) {
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= int64_t(ndof) * kNR) return;
  const int i = int(idx >> 4), rr = int(idx & 15);
  float z;
  if (dir[i]) {
    z = r[idx];
  } else {
    z = 0.f;
    for (int e = dptr[i]; e < dptr[i + 1]; ++e) z += delta[int64_t(e) * kNR + rr];
  }
  switch (mode) {
    case 0:
      zout[idx] = z;
      break;
    case 1: {
      const float dn = z / theta;
      d[idx] = dn;
      x[idx] = dn;
      break;
    }
    case 2: {
      const float dn = z / theta;
      d[idx] = dn;
      x[idx] += dn;
      break;
    }
    default: {
      const float dn = c1 * d[idx] + c2 * z;
      d[idx] = dn;
      x[idx] += dn;
      break;
    }
  }
}

// ---- coarse solve, FP32: X[n][16] = Minv[0:n,0:n] B[n][16], 32-row tiles, 64-wide k chunks ----------
__global__ void __launch_bounds__(512) k_coarse_mm(const float* __restrict__ Minv, int n, int ld,
                                                   const float* __restrict__ B, float* __restrict__ X) {
  __shared__ float As[32][65];
  __shared__ float Bs[64][kNR];
  const int tid = threadIdx.x;             // 512 threads: 32 rows x 16 rhs
  const int rl = tid >> 4, rr = tid & 15;
  const int row0 = blockIdx.x * 32;
  float acc = 0.f;
  for (int k0 = 0; k0 < n; k0 += 64) {
    for (int e = tid; e < 32 * 64; e += 512) {
      const int a = e >> 6, c = e & 63;
      const int row = row0 + a, k = k0 + c;
      As[a][c] = (row < n && k < n) ? Minv[int64_t(row) * ld + k] : 0.f;
    }
    for (int e = tid; e < 64 * kNR; e += 512) {
      const int c = e >> 4, q = e & 15, k = k0 + c;
      Bs[c][q] = k < n ? B[int64_t(k) * kNR + q] : 0.f;
    }
    __syncthreads();
#pragma unroll 16
    for (int c = 0; c < 64; ++c) acc = fmaf(As[rl][c], Bs[c][rr], acc);
    __syncthreads();
  }
  const int row = row0 + rl;
  if (row < n) X[int64_t(row) * kNR + rr] = acc;
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) b[i] = float(a[i]);
}

__global__ void k_to_f64(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) b[i] = double(a[i]);
}

// ---- FP64 block-vector helpers for the batched FGMRES ---------------------------------------------
// column-major (ld, nrhs columns) <-> interleaved [n][16]; missing columns are zero
__global__ void k_gather_cols(const double* __restrict__ B, int64_t ld, int nrhs, double* __restrict__ Y, int n) {
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= int64_t(n) * kNR) return;
  const int i = int(idx >> 4), r = int(idx & 15);
  Y[idx] = r < nrhs ? B[int64_t(r) * ld + i] : 0.0;
}

__global__ void k_scatter_cols(const double* __restrict__ Y, double* __restrict__ X, int64_t ld, int nrhs, int n) {
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= int64_t(n) * kNR) return;
  const int i = int(idx >> 4), r = int(idx & 15);
  if (r < nrhs) X[int64_t(r) * ld + i] = Y[idx];
}

// partial[(v * kNR + r) * nb + blockIdx.x] = sum over the block's rows of X_v[row][r] * W[row][r]
// for v < nvec (X_v = X + v * ldx).  Block = 256 threads = 16 rows x 16 rhs; grid-stride over rows.
__global__ void __launch_bounds__(kT) k_mdot_mm(const double* __restrict__ X, int64_t ldx, int nvec,
                                                const double* __restrict__ W, int lo, int len,
                                                double* __restrict__ partial, int nb) {
  __shared__ double sh[kT];
  const int rl = threadIdx.x >> 4, r = threadIdx.x & 15;
  for (int v = 0; v < nvec; ++v) {
    const double* x = X + ldx * v;
    double s = 0.0;
    for (int row = lo + blockIdx.x * 16 + rl; row < lo + len; row += nb * 16)
      s = fma(x[int64_t(row) * kNR + r], W[int64_t(row) * kNR + r], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kT / 2; o >= 16; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x < 16) partial[(int64_t(v) * kNR + threadIdx.x) * nb + blockIdx.x] = sh[threadIdx.x];
    __syncthreads();
  }
}

// out[v * kNR + r] = sum_b partial[(v * kNR + r) * nb + b]  (one block per (v, r)); acc adds
__global__ void __launch_bounds__(kT) k_mfin_mm(const double* __restrict__ partial, int nb, double* __restrict__ out,
                                                double* __restrict__ acc) {
  const int vr = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += kT) s += partial[int64_t(vr) * nb + b];
  s = block_sum_d<kT>(s);
  if (threadIdx.x == 0) {
    out[vr] = s;
    if (acc) acc[vr] += s;
  }
}

// W[row][r] -= sum_v X_v[row][r] * h[v * kNR + r]
__global__ void k_maxpy_mm(const double* __restrict__ X, int64_t ldx, int nvec, const double* __restrict__ h,
                           double* __restrict__ W, int n) {
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= int64_t(n) * kNR) return;
  const int r = int(idx & 15);
  double s = 0.0;
  for (int v = 0; v < nvec; ++v) s = fma(X[ldx * v + idx], h[v * kNR + r], s);
  W[idx] -= s;
}

// X[row][r] -= mean[r] on rows [lo, lo + len) where mean = sum[r] / len
__global__ void k_sub_mean_mm(double* __restrict__ X, int lo, int len, const double* __restrict__ sum) {
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= int64_t(len) * kNR) return;
  const int r = int(idx & 15);
  X[int64_t(lo) * kNR + idx] -= sum[r] / double(len);
}

// column sums over rows [lo, lo+len): partial[r * nb + b]
__global__ void __launch_bounds__(kT) k_colsum_mm(const double* __restrict__ X, int lo, int len,
                                                  double* __restrict__ partial, int nb) {
  __shared__ double sh[kT];
  const int rl = threadIdx.x >> 4, r = threadIdx.x & 15;
  double s = 0.0;
  for (int row = lo + blockIdx.x * 16 + rl; row < lo + len; row += nb * 16) s += X[int64_t(row) * kNR + r];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = kT / 2; o >= 16; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 16) partial[int64_t(threadIdx.x) * nb + blockIdx.x] = sh[threadIdx.x];
}

// Y[row][r] = active[r] && nrm[r] > 0 ? W[row][r] / nrm[r] : 0, nrm = sqrt(sq)
__global__ void k_normalize_mm(const double* __restrict__ W, const double* __restrict__ sq,
                               const int* __restrict__ active, double* __restrict__ Y, int n) {
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= int64_t(n) * kNR) return;
  const int r = int(idx & 15);
  const double nrm = sqrt(sq[r]);
  Y[idx] = (active[r] && nrm > 0.0) ? W[idx] / nrm : 0.0;
}

// X[row][r] = sum_{i < m[r]} y[r * ldy + i] Z_i[row][r]
__global__ void k_combine_mm(const double* __restrict__ Z, int64_t ldz, const int* __restrict__ m,
                             const double* __restrict__ y, int ldy, double* __restrict__ X, int n) {
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= int64_t(n) * kNR) return;
  const int r = int(idx & 15);
  double s = 0.0;
  for (int i = 0; i < m[r]; ++i) s = __dadd_rn(s, __dmul_rn(y[r * ldy + i], Z[ldz * i + idx]));
  X[idx] = s;
}

// Givens of column j for every active right-hand side (thread r): H_r column-major (ldh), estimates
// in hist[r * ldh + j + 1]; on convergence (or non-finite) clears active[r] and records iters[r].
__global__ void k_givens_mm(double* __restrict__ H, int ldh, int64_t hstride, double* __restrict__ cs,
                            double* __restrict__ sn, double* __restrict__ g, double* __restrict__ hist,
                            const double* __restrict__ hcol, const double* __restrict__ hnrm, int j, double rtol,
                            int* __restrict__ active, int* __restrict__ iters, int* __restrict__ nonfinite) {
  const int r = threadIdx.x;
  if (r >= kNR || !active[r]) return;
  double* h = H + hstride * r + int64_t(j) * ldh;
  for (int i = 0; i <= j; ++i) h[i] = hcol[i * kNR + r];
  h[j + 1] = sqrt(hnrm[r]);
  double* c = cs + int64_t(r) * ldh;
  double* s = sn + int64_t(r) * ldh;
  double* gg = g + int64_t(r) * ldh;
  for (int i = 0; i < j; ++i) {
    const double t = __dadd_rn(__dmul_rn(c[i], h[i]), __dmul_rn(s[i], h[i + 1]));
    h[i + 1] = __dadd_rn(__dmul_rn(-s[i], h[i]), __dmul_rn(c[i], h[i + 1]));
    h[i] = t;
  }
  const double den = hypot(h[j], h[j + 1]);
  const double cj = h[j] / den, sj = h[j + 1] / den;
  c[j] = cj;
  s[j] = sj;
  h[j] = den;
  h[j + 1] = 0.0;
  gg[j + 1] = -sj * gg[j];
  gg[j] = cj * gg[j];
  const double est = fabs(gg[j + 1]);
  hist[int64_t(r) * ldh + j + 1] = est;
  iters[r] = j + 1;
  if (!isfinite(est)) {
    nonfinite[r] = 1;
    active[r] = 0;
  } else if (est <= rtol * hist[int64_t(r) * ldh]) {
    active[r] = 0;
  }
}

}  // namespace

// ---- launchers ------------------------------------------------------------------------------------
template <typename T>
int mm_csr(const Csr& A, const T* val, int mode, const T* b, const uint8_t* mask, const T* x, T* y,
           cudaStream_t s) {
  if (A.nrows == 0) return 0;
  const int g = nblk(int64_t(A.nrows) * 16);
  switch (mode) {
    case 0: k_mm<T, 0><<<g, kT, 0, s>>>(A.nrows, A.ptr, A.col, val, b, mask, x, y); break;
    case 1: k_mm<T, 1><<<g, kT, 0, s>>>(A.nrows, A.ptr, A.col, val, b, mask, x, y); break;
    case 2: k_mm<T, 2><<<g, kT, 0, s>>>(A.nrows, A.ptr, A.col, val, b, mask, x, y); break;
    default: k_mm<T, 3><<<g, kT, 0, s>>>(A.nrows, A.ptr, A.col, val, b, mask, x, y); break;
  }
  return 1;
}
template int mm_csr<float>(const Csr&, const float*, int, const float*, const uint8_t*, const float*, float*,
                           cudaStream_t);
template int mm_csr<double>(const Csr&, const double*, int, const double*, const uint8_t*, const double*, double*,
                            cudaStream_t);

int pack_mma(const Patches& P, const double* inv64, const int64_t* foff16, void* frag, float* ascale, bool half,
             cudaStream_t s) {
  if (P.npatch == 0) return 0;
  if (half)
    k_pack_mma<true><<<P.npatch, 128, 0, s>>>(P.slot_ptr, P.foff, inv64, foff16, static_cast<uint4*>(frag), ascale);
  else
    k_pack_mma<false><<<P.npatch, 128, 0, s>>>(P.slot_ptr, P.foff, inv64, foff16, static_cast<uint4*>(frag), ascale);
  return 1;
}

int patch_apply_mma(const Patches& P, const int64_t* foff16, const void* frag, const float* ascale, bool half,
                    int mt_max, const float* rhs, float* delta, cudaStream_t s) {
  if (P.npatch == 0) return 0;
  const int blocks = (P.npatch + 7) / 8;
  const uint4* f = static_cast<const uint4*>(frag);
#define VK_MMA_LAUNCH(MTM)                                                                                   \
  do {                                                                                                       \
    if (half)                                                                                                \
      k_patch_mma<MTM, true><<<blocks, kT, 0, s>>>(P.npatch, P.work, P.slot_ptr, P.slot_dofs, foff16, f,     \
                                                   ascale, rhs, P.slot_pos, delta);                          \
    else                                                                                                     \
      k_patch_mma<MTM, false><<<blocks, kT, 0, s>>>(P.npatch, P.work, P.slot_ptr, P.slot_dofs, foff16, f,    \
                                                    ascale, rhs, P.slot_pos, delta);                         \
  } while (0)
  if (mt_max <= 3)
    VK_MMA_LAUNCH(3);
  else if (mt_max <= 5)
    VK_MMA_LAUNCH(5);
  else
    VK_MMA_LAUNCH(8);
#undef VK_MMA_LAUNCH
  return 1;
}

int scatter_mm(const Patches& P, int ndof, const uint8_t* dir, const float* r, const float* delta, int mode,
               float theta, float c1, float c2, float* zout, float* d, float* x, cudaStream_t s) {
  k_scatter_mm<<<nblk(int64_t(ndof) * 16), kT, 0, s>>>(ndof, P.dof_ptr, dir, r, delta, mode, theta, c1, c2, zout, d,
                                                        x);
  return 1;
}

int coarse_mm(const float* Minv, int n, int ld, const float* B, float* X, cudaStream_t s) {
  k_coarse_mm<<<(n + 31) / 32, 512, 0, s>>>(Minv, n, ld, B, X);
  return 1;
}

int to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  k_to_f32<<<nblk(n), kT, 0, s>>>(a, b, n);
  return 1;
}

int to_f64(const float* a, double* b, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  k_to_f64<<<nblk(n), kT, 0, s>>>(a, b, n);
  return 1;
}

int gather_cols(const double* B, int64_t ld, int nrhs, double* Y, int n, cudaStream_t s) {
  k_gather_cols<<<nblk(int64_t(n) * 16), kT, 0, s>>>(B, ld, nrhs, Y, n);
  return 1;
}

int scatter_cols(const double* Y, double* X, int64_t ld, int nrhs, int n, cudaStream_t s) {
  k_scatter_cols<<<nblk(int64_t(n) * 16), kT, 0, s>>>(Y, X, ld, nrhs, n);
  return 1;
}

constexpr int kBatchBlocks = 256;

int mdot_mm(const double* X, int64_t ldx, int nvec, const double* W, int n, double* partial, double* out,
            double* acc, cudaStream_t s) {
  if (nvec <= 0) return 0;
  k_mdot_mm<<<kBatchBlocks, kT, 0, s>>>(X, ldx, nvec, W, 0, n, partial, kBatchBlocks);
  k_mfin_mm<<<nvec * 16, kT, 0, s>>>(partial, kBatchBlocks, out, acc);
  return 2;
}

int maxpy_mm(const double* X, int64_t ldx, int nvec, const double* h, double* W, int n, cudaStream_t s) {
  k_maxpy_mm<<<nblk(int64_t(n) * 16), kT, 0, s>>>(X, ldx, nvec, h, W, n);
  return 1;
}

int project_mm(double* X, int lo, int len, double* partial, double* sum, cudaStream_t s) {
  if (len <= 0) return 0;
  k_colsum_mm<<<kBatchBlocks, kT, 0, s>>>(X, lo, len, partial, kBatchBlocks);
  k_mfin_mm<<<16, kT, 0, s>>>(partial, kBatchBlocks, sum, nullptr);
  k_sub_mean_mm<<<nblk(int64_t(len) * 16), kT, 0, s>>>(X, lo, len, sum);
  return 3;
}

int normalize_mm(const double* W, const double* sq, const int* active, double* Y, int n, cudaStream_t s) {
  k_normalize_mm<<<nblk(int64_t(n) * 16), kT, 0, s>>>(W, sq, active, Y, n);
  return 1;
}

int combine_mm(const double* Z, int64_t ldz, const int* m, const double* y, int ldy, double* X, int n,
               cudaStream_t s) {
  k_combine_mm<<<nblk(int64_t(n) * 16), kT, 0, s>>>(Z, ldz, m, y, ldy, X, n);
  return 1;
}

int givens_mm(double* H, int ldh, int64_t hstride, double* cs, double* sn, double* g, double* hist,
              const double* hcol, const double* hnrm, int j, double rtol, int* active, int* iters, int* nonfinite,
              cudaStream_t s) {
  k_givens_mm<<<1, 32, 0, s>>>(H, ldh, hstride, cs, sn, g, hist, hcol, hnrm, j, rtol, active, iters, nonfinite);
  return 1;
}

}  // namespace gpu
}  // namespace vk
