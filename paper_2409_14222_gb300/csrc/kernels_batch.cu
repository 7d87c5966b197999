// Multi-right-hand-side kernels (vk_solve_batch): block vectors hold kNR = 16 right-hand sides
// interleaved per DoF ([ndof][16], the 16 values of a DoF are contiguous), so a matrix entry is read
// once for 16 products and a gathered row is one 64-byte (FP32) or 128-byte (FP64) access.
//
// The V-cycle preconditioner runs in FP32 (FP32 matrices, FP32 block vectors); the patch solves of
// Algorithm 1 become a dense contraction delta_i[n x 16] = A_i^{-1}[n x n] R_i[n x 16] per patch,
// done on the tensor cores with 16-bit inputs (BF16 or FP16) and FP32 accumulation: mma.sync
// m16n8k16 here, tcgen05 in kernels_tc.cu.  A_i^{-1} is stored scaled by its largest magnitude,
// pre-packed in the A-fragment order of the instruction (one 16-byte load per lane per 16x16 tile);
// with FP16 each right-hand-side column of R_i is scaled by its own largest magnitude over the patch
// (FP16's exponent range), with BF16 (FP32's exponent range) the columns are rounded as they are.
// Either way a column's result does not depend on the other columns.
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

// ---- block SpMM, SELL-8 (slices of 8 rows, rows sorted by length in windows) ---------------------
//   kMode as k_mm.  Warp = one slice: lane 4 t + q owns row t of the slice and right-hand sides
//   4q .. 4q+3, and walks all entries of its row in order (entry m of row t at sptr + 8 m + t, so a
//   warp load of columns or values is 8 consecutive entries); the x rows of kU entries are loaded
//   before their products, 8 rows x 64 (FP32) or 128 (FP64) contiguous bytes per load instruction.
//   Padding entries have value 0 and a valid column.  Each row is summed in its CSR order, exactly
//   like the sequential loop of k_mm.
template <typename T>
struct Vec4 {
  T v[4];
};
__device__ __forceinline__ Vec4<float> ld4(const float* p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Vec4<double> ld4(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ Vec4<float> ld4_plain(const float* p) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Vec4<double> ld4_plain(const double* p) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *(reinterpret_cast<const double2*>(p) + 1);
  return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, const Vec4<float>& a) {
  *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}
__device__ __forceinline__ void st4(double* p, const Vec4<double>& a) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a.v[0], a.v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(a.v[2], a.v[3]);
}

template <typename T, int kMode>
__global__ void __launch_bounds__(kT) k_sell_mm(int nslices, const int64_t* __restrict__ sptr,
                                                const int* __restrict__ sw, const int* __restrict__ col,
                                                const T* __restrict__ val, const int* __restrict__ rowof,
                                                const T* b, const uint8_t* __restrict__ mask,
                                                const T* __restrict__ x, T* y) {
  constexpr int kU = sizeof(T) == 4 ? 8 : 4;
  const int warp = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= nslices) return;
  const int t = lane >> 2, q = lane & 3;
  const int row = rowof[warp * 8 + t];
  const int w = sw[warp];
  const int64_t base = sptr[warp] + t;
  Vec4<T> acc = {{T(0), T(0), T(0), T(0)}};
  int m = 0;
  for (; m + kU <= w; m += kU) {
    int c[kU];
    T v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      c[u] = __ldg(col + base + 8 * int64_t(m + u));
      v[u] = __ldg(val + base + 8 * int64_t(m + u));
    }
    Vec4<T> xv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) xv[u] = ld4(x + int64_t(c[u]) * kNR + 4 * q);
#pragma unroll
    for (int u = 0; u < kU; ++u)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc.v[e] = fma(v[u], xv[u].v[e], acc.v[e]);
  }
  for (; m < w; ++m) {
    const int c = __ldg(col + base + 8 * int64_t(m));
    const T v = __ldg(val + base + 8 * int64_t(m));
    const Vec4<T> xv = ld4(x + int64_t(c) * kNR + 4 * q);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc.v[e] = fma(v, xv.v[e], acc.v[e]);
  }
  if (row < 0) return;
  T* o = y + int64_t(row) * kNR + 4 * q;
  Vec4<T> r;
  if (kMode == 0 || kMode == 2) {
    const Vec4<T> bb = ld4_plain(b + int64_t(row) * kNR + 4 * q);
#pragma unroll
    for (int e = 0; e < 4; ++e) r.v[e] = kMode == 0 ? bb.v[e] - acc.v[e] : bb.v[e] + acc.v[e];
  } else if (kMode == 1) {
    r = acc;
  } else {
    const bool z = mask[row] != 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) r.v[e] = z ? T(0) : acc.v[e];
  }
  st4(o, r);
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
  // per-column scale (FP16 only: its 5-bit exponent needs the column in range; BF16 keeps FP32's
  // exponent range, so its columns are rounded unscaled): lanes 4g .. 4g+3 hold the rows of column
  // nt*8 + g
  if constexpr (kHalf) {
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      cmax[nt] = fmaxf(cmax[nt], __shfl_xor_sync(0xffffffffu, cmax[nt], 1));
      cmax[nt] = fmaxf(cmax[nt], __shfl_xor_sync(0xffffffffu, cmax[nt], 2));
    }
  } else {
    cmax[0] = cmax[1] = 1.f;
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
    const int e0 = dptr[i], e1 = dptr[i + 1];
    // the first 8 corrections as one predicated batch (all loads in flight), the rest in order
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = e0 + u < e1 ? delta[int64_t(e0 + u) * kNR + rr] : 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (e0 + u < e1) z += v[u];
    for (int e = e0 + 8; e < e1; ++e) z += delta[int64_t(e) * kNR + rr];
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

// ---- coarse solve, FP32: X[n][16] = Minv[0:n,0:n] B[n][16] ------------------------------------
// Block = 16 rows x 16 right-hand sides (thread (row, rhs)); k runs in chunks of 128: the A tile
// (16 x 128, row-major rows of Minv, float4 loads) and the B tile (128 x 16) are staged in shared
// memory, the next chunk's loads are issued into registers before the current chunk's products.
constexpr int kCoarseRows = 16, kCoarseK = 128;
__global__ void __launch_bounds__(256) k_coarse_mm(const float* __restrict__ Minv, int n, int ld,
                                                   const float* __restrict__ B, float* __restrict__ X) {
  __shared__ float4 As[kCoarseRows][kCoarseK / 4 + 1];
  __shared__ float Bs[kCoarseK][kNR];
  const int tid = threadIdx.x;
  const int rl = tid >> 4, rr = tid & 15;
  const int row0 = blockIdx.x * kCoarseRows;
  // loader roles: 2 float4 of A (row tid / 16 ... ) and 2 float4 of B per thread and chunk
  float4 pa[2], pb[2];
  auto load = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + 256 * u;                  // 0..511: A tile as 16 rows x 32 float4
      const int ar = e >> 5, ac = (e & 31) * 4;
      const int row = row0 + ar, k = k0 + ac;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < n) {
        const float* src = Minv + int64_t(row) * ld + k;
        if (k + 3 < n && (((reinterpret_cast<uintptr_t>(src)) & 15) == 0)) {
          v = __ldg(reinterpret_cast<const float4*>(src));
        } else {
          v.x = k < n ? src[0] : 0.f;
          v.y = k + 1 < n ? src[1] : 0.f;
          v.z = k + 2 < n ? src[2] : 0.f;
          v.w = k + 3 < n ? src[3] : 0.f;
        }
      }
      pa[u] = v;
      const int bk = e >> 2, bq = (e & 3) * 4;        // B tile as 128 rows x 4 float4
      pb[u] = (k0 + bk < n) ? __ldg(reinterpret_cast<const float4*>(B + int64_t(k0 + bk) * kNR + bq))
                            : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  float acc = 0.f;
  load(0);
  for (int k0 = 0; k0 < n; k0 += kCoarseK) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + 256 * u;
      As[e >> 5][e & 31] = pa[u];
      *reinterpret_cast<float4*>(&Bs[e >> 2][(e & 3) * 4]) = pb[u];
    }
    __syncthreads();
    if (k0 + kCoarseK < n) load(k0 + kCoarseK);
#pragma unroll 8
    for (int c = 0; c < kCoarseK / 4; ++c) {
      const float4 a = As[rl][c];
      acc = fmaf(a.x, Bs[4 * c][rr], acc);
      acc = fmaf(a.y, Bs[4 * c + 1][rr], acc);
      acc = fmaf(a.z, Bs[4 * c + 2][rr], acc);
      acc = fmaf(a.w, Bs[4 * c + 3][rr], acc);
    }
  }
  const int row = row0 + rl;
  if (row < n) X[int64_t(row) * kNR + rr] = acc;
}

// ---- coarse solve, FP64: X[n][16] = Minv[0:n,0:n] B[n][16] --------------------------------------
// Same blocking as k_coarse_mm (16 rows x 16 right-hand sides per block) with 64-wide K chunks of
// doubles; the next chunk's loads are issued into registers before the current chunk's products.
constexpr int kCoarseK64 = 64;
__global__ void __launch_bounds__(256) k_coarse_mm64(const double* __restrict__ Minv, int n, int ld,
                                                     const double* __restrict__ B, double* __restrict__ X) {
  __shared__ double2 As[kCoarseRows][kCoarseK64 / 2 + 1];
  __shared__ double Bs[kCoarseK64][kNR];
  const int tid = threadIdx.x;
  const int rl = tid >> 4, rr = tid & 15;
  const int row0 = blockIdx.x * kCoarseRows;
  double2 pa[2], pb[2];
  auto load = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + 256 * u;                  // 0..511: A tile as 16 rows x 32 double2
      const int ar = e >> 5, ac = (e & 31) * 2;
      const int row = row0 + ar, k = k0 + ac;
      double2 v = make_double2(0.0, 0.0);
      if (row < n) {
        const double* src = Minv + int64_t(row) * ld + k;
        v.x = k < n ? src[0] : 0.0;
        v.y = k + 1 < n ? src[1] : 0.0;
      }
      pa[u] = v;
      const int bk = e >> 3, bq = (e & 7) * 2;        // B tile as 64 rows x 8 double2
      pb[u] = (k0 + bk < n) ? *reinterpret_cast<const double2*>(B + int64_t(k0 + bk) * kNR + bq)
                            : make_double2(0.0, 0.0);
    }
  };
  double acc = 0.0;
  load(0);
  for (int k0 = 0; k0 < n; k0 += kCoarseK64) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + 256 * u;
      As[e >> 5][e & 31] = pa[u];
      *reinterpret_cast<double2*>(&Bs[e >> 3][(e & 7) * 2]) = pb[u];
    }
    __syncthreads();
    if (k0 + kCoarseK64 < n) load(k0 + kCoarseK64);
#pragma unroll 8
    for (int c = 0; c < kCoarseK64 / 2; ++c) {
      const double2 a = As[rl][c];
      acc = fma(a.x, Bs[2 * c][rr], acc);
      acc = fma(a.y, Bs[2 * c + 1][rr], acc);
    }
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
// for v < nvec (X_v = X + v * ldx).  Thread t of a block always handles right-hand side t % 16 (the
// grid stride is a multiple of 16); the vectors are taken kVB at a time, so W is read once per kVB
// vectors and kVB + 1 independent loads are in flight per element.  Fixed reduction tree: lanes
// (r, r + 16) of a warp, then the 8 warps in order.
constexpr int kVB = 8;
__global__ void __launch_bounds__(kT) k_mdot_mm(const double* __restrict__ X, int64_t ldx, int nvec,
                                                const double* __restrict__ W, int64_t n16,
                                                double* __restrict__ partial, int nb) {
  __shared__ double sh[kT / 32][kVB][16];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int v0 = 0; v0 < nvec; v0 += kVB) {
    double acc[kVB];
#pragma unroll
    for (int u = 0; u < kVB; ++u) acc[u] = 0.0;
    // four grid strides per step: 4 (kVB + 1) independent loads in flight per thread
    const int64_t stride = int64_t(nb) * kT;
    int64_t idx = int64_t(blockIdx.x) * kT + tid;
    for (; idx + 3 * stride < n16; idx += 4 * stride) {
      double w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) w[e] = W[idx + e * stride];
#pragma unroll
      for (int u = 0; u < kVB; ++u)
        if (v0 + u < nvec) {
          const double* x = X + ldx * (v0 + u) + idx;
          const double x0 = x[0], x1 = x[stride], x2 = x[2 * stride], x3 = x[3 * stride];
          acc[u] = fma(x0, w[0], acc[u]);
          acc[u] = fma(x1, w[1], acc[u]);
          acc[u] = fma(x2, w[2], acc[u]);
          acc[u] = fma(x3, w[3], acc[u]);
        }
    }
    for (; idx < n16; idx += stride) {
      const double w = W[idx];
#pragma unroll
      for (int u = 0; u < kVB; ++u)
        if (v0 + u < nvec) acc[u] = fma(X[ldx * (v0 + u) + idx], w, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < kVB; ++u) {
      const double t = acc[u] + __shfl_xor_sync(0xffffffffu, acc[u], 16);
      if (lane < 16) sh[warp][u][lane] = t;
    }
    __syncthreads();
    if (tid < kVB * 16) {
      const int u = tid >> 4, r = tid & 15;
      if (v0 + u < nvec) {
        double sum = 0.0;
#pragma unroll
        for (int w8 = 0; w8 < kT / 32; ++w8) sum += sh[w8][u][r];
        partial[(int64_t(v0 + u) * kNR + r) * nb + blockIdx.x] = sum;
      }
    }
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

// W[row][r] -= sum_v X_v[row][r] * h[v * kNR + r], summed in ascending v.  Each thread takes four
// elements one block-width apart (same right-hand side r), so four independent loads are in flight
// for every vector even when there are only a few vectors.
constexpr int kAxpyE = 4;
__global__ void __launch_bounds__(kT) k_maxpy_mm(const double* __restrict__ X, int64_t ldx, int nvec,
                                                 const double* __restrict__ h, double* __restrict__ W, int64_t n16) {
  const int64_t base = int64_t(blockIdx.x) * kT * kAxpyE + threadIdx.x;
  const int r = threadIdx.x & 15;
  double s[kAxpyE];
#pragma unroll
  for (int e = 0; e < kAxpyE; ++e) s[e] = 0.0;
#pragma unroll 4
  for (int v = 0; v < nvec; ++v) {
    const double hv = __ldg(h + v * kNR + r);
    const double* x = X + ldx * v + base;
#pragma unroll
    for (int e = 0; e < kAxpyE; ++e)
      if (base + e * kT < n16) s[e] = fma(x[e * kT], hv, s[e]);
  }
#pragma unroll
  for (int e = 0; e < kAxpyE; ++e)
    if (base + e * kT < n16) W[base + e * kT] -= s[e];
}

// X[row][r] -= mean[r] on rows [lo, lo + len) where mean = sum[r] / len (16 divisions per block)
__global__ void k_sub_mean_mm(double* __restrict__ X, int lo, int len, const double* __restrict__ sum) {
  __shared__ double mean[kNR];
  if (threadIdx.x < kNR) mean[threadIdx.x] = sum[threadIdx.x] / double(len);
  __syncthreads();
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= int64_t(len) * kNR) return;
  X[int64_t(lo) * kNR + idx] -= mean[idx & 15];
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

// Y[row][r] = active[r] && nrm[r] > 0 ? W[row][r] * (1 / nrm[r]) : 0, nrm = sqrt(sq): the 16
// reciprocals are formed once per block
__global__ void k_normalize_mm(const double* __restrict__ W, const double* __restrict__ sq,
                               const int* __restrict__ active, double* __restrict__ Y, int n) {
  __shared__ double inv[kNR];
  if (threadIdx.x < kNR) {
    const double nrm = sqrt(sq[threadIdx.x]);
    inv[threadIdx.x] = (active[threadIdx.x] && nrm > 0.0) ? 1.0 / nrm : 0.0;
  }
  __syncthreads();
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= int64_t(n) * kNR) return;
  Y[idx] = W[idx] * inv[idx & 15];
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
int mm_sell(const SellB& A, const T* val, int mode, const T* b, const uint8_t* mask, const T* x, T* y,
            cudaStream_t s) {
  if (A.nslices == 0) return 0;
  const int g = nblk(int64_t(A.nslices) * 32);
  switch (mode) {
    case 0: k_sell_mm<T, 0><<<g, kT, 0, s>>>(A.nslices, A.sptr, A.swidth, A.col, val, A.rowof, b, mask, x, y); break;
    case 1: k_sell_mm<T, 1><<<g, kT, 0, s>>>(A.nslices, A.sptr, A.swidth, A.col, val, A.rowof, b, mask, x, y); break;
    case 2: k_sell_mm<T, 2><<<g, kT, 0, s>>>(A.nslices, A.sptr, A.swidth, A.col, val, A.rowof, b, mask, x, y); break;
    default: k_sell_mm<T, 3><<<g, kT, 0, s>>>(A.nslices, A.sptr, A.swidth, A.col, val, A.rowof, b, mask, x, y); break;
  }
  return 1;
}
template int mm_sell<float>(const SellB&, const float*, int, const float*, const uint8_t*, const float*, float*,
                            cudaStream_t);
template int mm_sell<double>(const SellB&, const double*, int, const double*, const uint8_t*, const double*, double*,
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
  k_coarse_mm<<<(n + kCoarseRows - 1) / kCoarseRows, 256, 0, s>>>(Minv, n, ld, B, X);
  return 1;
}

int coarse_mm64(const double* Minv, int n, int ld, const double* B, double* X, cudaStream_t s) {
  k_coarse_mm64<<<(n + kCoarseRows - 1) / kCoarseRows, 256, 0, s>>>(Minv, n, ld, B, X);
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

int mdot_mm(const double* X, int64_t ldx, int nvec, const double* W, int n, double* partial, double* out,
            double* acc, cudaStream_t s) {
  if (nvec <= 0) return 0;
  k_mdot_mm<<<kBatchBlocks, kT, 0, s>>>(X, ldx, nvec, W, int64_t(n) * kNR, partial, kBatchBlocks);
  k_mfin_mm<<<nvec * 16, kT, 0, s>>>(partial, kBatchBlocks, out, acc);
  return 2;
}

int maxpy_mm(const double* X, int64_t ldx, int nvec, const double* h, double* W, int n, cudaStream_t s) {
  k_maxpy_mm<<<nblk(int64_t(n) * 16, kT * kAxpyE), kT, 0, s>>>(X, ldx, nvec, h, W, int64_t(n) * kNR);
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
