// Vanka patch kernels (Sec. 3.1, Algorithm 1):
//   patch_factor  -- gather A_i = A[idx_i, idx_i] from the assembled CSR matrix (matrix-full,
//                    Sec. 3.1 last paragraph) and invert it in shared memory by Gauss-Jordan
//                    elimination with partial pivoting; store the inverse in the warp-packed layout.
//   patch_apply   -- delta_i = A_i^{-1} r[idx_i] for every patch: one warp per patch, in one launch
//                    or one launch per size class, with the launch shape the setup autotuner chose.
//   vanka_scatter -- z_d = sum over the patches i containing DoF d of (w_d delta_i)_d, summed in
//                    ascending patch order (atomic-free), Dirichlet identity, fused with the
//                    Chebyshev update of Sec. 3 ("Relaxation").
//
// Warp-packed layout of an n x n inverse: NA = ceil(n/8) row blocks, NB = ceil(n/4) column steps.
// Lane l = r + 8 c (r in 0..7, c in 0..3) owns rows r + 8 a and columns c + 4 b.  Element (a, b) of
// lane l is stored at (a * NB + b) * 32 + l, so each warp load is 32 consecutive values (256 bytes in
// FP64), and padding (rows/columns >= n, stored as zero) is at most 7 rows and 3 columns.
#include <algorithm>
#include <cfloat>
#include <type_traits>

#include "gpu.h"

namespace vk {
namespace gpu {

namespace {

constexpr int kFactorThreads = 128;

template <typename FT>
__device__ __forceinline__ FT store_entry(double v) {
  return FT(v);
}
// FP32 pair: hi = fl32(v), lo = fl32(v - hi); hi + lo carries 48 significant bits of v
template <>
__device__ __forceinline__ float2 store_entry<float2>(double v) {
  const float hi = __double2float_rn(v);
  const float lo = __double2float_rn(v - double(hi));
  return make_float2(hi, lo);
}

template <typename FT, bool kMF>
__global__ void __launch_bounds__(kFactorThreads) k_patch_factor(Csr A, PatchElems E, const int* __restrict__ slot_ptr,
                                                                 const int* __restrict__ slot_dofs,
                                                                 const int64_t* __restrict__ foff,
                                                                 FT* __restrict__ F, int* status, int sym) {
  extern __shared__ double sm[];
  __shared__ double red_v[kFactorThreads / 32];
  __shared__ int red_i[kFactorThreads / 32];
  __shared__ int piv_row, bad;
  const int p = blockIdx.x, tid = threadIdx.x;
  const int s0 = slot_ptr[p], n = slot_ptr[p + 1] - s0;
  const int* dofs = slot_dofs + s0;
  double* M = sm;              // n * n, row-major
  double* fcol = M + n * n;    // n
  int* perm = reinterpret_cast<int*>(fcol + n);  // n
  for (int i = tid; i < n * n; i += kFactorThreads) M[i] = 0.0;
  __syncthreads();
  auto find = [&](int c) {   // position of global DoF c in the sorted patch list, or -1
    int lo = 0, hi = n;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (dofs[mid] < c) lo = mid + 1; else hi = mid;
    }
    return (lo < n && dofs[lo] == c) ? lo : -1;
  };
  if (!kMF) {
    // matrix-full gather: row i of the patch scans CSR row dofs[i]; each column is located in the
    // sorted list
    for (int i = tid; i < n; i += kFactorThreads) {
      const int g = dofs[i];
      for (int e = A.ptr[g]; e < A.ptr[g + 1]; ++e) {
        const int j = find(A.col[e]);
        if (j >= 0) M[i * n + j] = A.val[e];
      }
    }
  } else {
    // matrix-free assembly: row i sums, over the patch's cells in ascending order, the element-matrix
    // row of its DoF into the patch columns (each cell is visited again by every patch it serves)
    for (int i = tid; i < n; i += kFactorThreads) {
      const int g = dofs[i];
      for (int t = E.cell_ptr[p]; t < E.cell_ptr[p + 1]; ++t) {
        const int c = E.cells[t];
        const int* cd = E.cell_dofs + int64_t(c) * E.nloc;
        int la = -1;
        for (int q = 0; q < E.nloc; ++q)
          if (cd[q] == g) {
            la = q;
            break;
          }
        if (la < 0) continue;
        const double* K = E.kel + (int64_t(c < E.ncell_lower ? 0 : 1) * E.nloc + la) * E.nloc;
        for (int q = 0; q < E.nloc; ++q) {
          const int j = find(cd[q]);
          if (j >= 0) M[i * n + j] += K[q];
        }
      }
    }
  }
  __syncthreads();
  // in-place Gauss-Jordan with partial pivoting (first maximal |pivot| wins ties)
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = n;
    for (int i = k + tid; i < n; i += kFactorThreads) {
      const double v = fabs(M[i * n + k]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = red_v[0];
      int bidx = red_i[0];
      for (int w = 1; w < kFactorThreads / 32; ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bidx)) { bv = red_v[w]; bidx = red_i[w]; }
      piv_row = bidx;
      bad = !(bv > 0.0) || !isfinite(bv);
      perm[k] = bidx;
    }
    __syncthreads();
    if (bad) {
      if (tid == 0) atomicCAS(status, 0, p + 1);
      return;
    }
    const int pr = piv_row;
    if (pr != k)
      for (int j = tid; j < n; j += kFactorThreads) {
        const double t = M[k * n + j];
        M[k * n + j] = M[pr * n + j];
        M[pr * n + j] = t;
      }
    __syncthreads();
    const double pv = M[k * n + k];
    for (int i = tid; i < n; i += kFactorThreads) fcol[i] = M[i * n + k];
    __syncthreads();
    for (int j = tid; j < n; j += kFactorThreads) M[k * n + j] = (j == k ? 1.0 : M[k * n + j]) / pv;
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += kFactorThreads) {
      const int i = idx / n, j = idx - i * n;
      if (i == k) continue;
      M[idx] = (j == k ? 0.0 : M[idx]) - fcol[i] * M[k * n + j];
    }
    __syncthreads();
  }
  // undo the row interchanges on the columns, last interchange first
  for (int i = tid; i < n; i += kFactorThreads)
    for (int k = n - 1; k >= 0; --k) {
      const int q = perm[k];
      if (q != k) {
        const double t = M[i * n + k];
        M[i * n + k] = M[i * n + q];
        M[i * n + q] = t;
      }
    }
  __syncthreads();
  FT* out = F + foff[p];
  if (sym) {
    // symmetric tile layout: tiles (I, J), I <= J, row-major; entry (i, j + 4 w) of a tile at 2 l + w
    // with l = i + 8 j; the stored value is the mean of the two mirrored entries
    const int NT = (n + 7) / 8;
    for (int e = tid; e < 32 * NT * (NT + 1); e += kFactorThreads) {
      int rem = e >> 6, I = 0;
      while (rem >= NT - I) {
        rem -= NT - I;
        ++I;
      }
      const int J = I + rem, l = (e & 63) >> 1, w = e & 1;
      const int row = 8 * I + (l & 7), col = 8 * J + (l >> 3) + 4 * w;
      out[e] = store_entry<FT>((row < n && col < n) ? 0.5 * (M[row * n + col] + M[col * n + row]) : 0.0);
    }
    return;
  }
  const int NB = (n + 3) / 4, NA = (n + 7) / 8;
  for (int e = tid; e < 32 * NA * NB; e += kFactorThreads) {
    const int lane = e & 31, ab = e >> 5;
    const int a = ab / NB, b = ab - a * NB;
    const int row = (lane & 7) + 8 * a, col = (lane >> 3) + 4 * b;
    out[e] = store_entry<FT>((row < n && col < n) ? M[row * n + col] : 0.0);
  }
}

template <typename FT>
struct Compute {
  using T = double;
};
template <>
struct Compute<float> {
  using T = float;
};

// One warp applies one packed inverse.  FP64 factors: FP64 products and sums.  FP32 factors: the
// local residual is rounded to FP32 and the products are summed in FP32.
template <int NB, typename FT>
__device__ __forceinline__ void apply_one(int n, int s0, const int* __restrict__ dofs,
                                          const FT* __restrict__ Fp, const double* __restrict__ r,
                                          const int* __restrict__ pos, double* __restrict__ delta, int lane) {
  using T = typename Compute<FT>::T;
  constexpr int NA = (NB + 1) / 2;
  const int rr = lane & 7, cc = lane >> 3;
  T rl[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = cc + 4 * b;
    rl[b] = j < n ? T(r[__ldg(dofs + j)]) : T(0);
  }
  T acc[NA];
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    T s = T(0);
#pragma unroll
    for (int b = 0; b < NB; ++b) s = fma(T(__ldg(Fp + (a * NB + b) * 32 + lane)), rl[b], s);
    acc[a] = s;
  }
  // Reduce-scatter of the four column-group partial sums (lanes cc = 0..3 of row set rr): the pair
  // (cc, cc ^ 2) splits the NA row blocks into halves and each lane adds only the half it keeps, then
  // the pair (cc, cc ^ 1) does the same on that half.  NA/2 + NA/4 additions per lane instead of the
  // 2 NA of a butterfly, which matters when the FP64 pipe is the bound; every lane ends with up to H2
  // finished rows and writes them.
  constexpr int H1 = (NA + 1) / 2, H2 = (H1 + 1) / 2;
  const bool h1 = (cc >> 1) != 0, h2 = (cc & 1) != 0;
  T b1[H1];
#pragma unroll
  for (int i = 0; i < H1; ++i) {
    const T lo = acc[i];
    const T hi = (H1 + i < NA) ? acc[H1 + i < NA ? H1 + i : 0] : T(0);
    const T send = h1 ? lo : hi, keep = h1 ? hi : lo;
    b1[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < H2; ++i) {
    const T lo = b1[i];
    const T hi = (H2 + i < H1) ? b1[H2 + i < H1 ? H2 + i : 0] : T(0);
    const T send = h2 ? lo : hi, keep = h2 ? hi : lo;
    const T v = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    const int a = (h1 ? H1 : 0) + (h2 ? H2 : 0) + i;
    const int row = rr + 8 * a;
    if ((h2 ? H2 : 0) + i < H1 && a < NA && row < n) delta[__ldg(pos + s0 + row)] = double(v);
  }
}

// FP32-pair (emulated FP64) apply.  The inverse entry a = ah + al and the local residual
// r = rh + rl (split once per DoF by k_split_pairs) are FP32 pairs; each product is
// p = fl(ah*rh), e = (ah*rh - p) + ah*rl + al*rh (first term exact by FMA); p is accumulated with
// TwoSum into (hi, err) and the low-order terms into lo, so row sums carry ~48 bits.  The cross-lane
// reduction stays in pair arithmetic and the corrections are written as pairs: no FP64 instruction
// runs per patch (FP64 is 1/64 of the FP32 rate on this part).  Every operation is an explicitly
// rounded intrinsic, so no contraction or reassociation can break the error-free transformations.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float p) {
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

template <int NB>
__device__ __forceinline__ void apply_one_pair(int n, int s0, const int* __restrict__ dofs,
                                               const float2* __restrict__ Fp, const float2* __restrict__ r2,
                                               const int* __restrict__ pos, float2* __restrict__ delta, int lane) {
  constexpr int NA = (NB + 1) / 2;
  const int rr = lane & 7, cc = lane >> 3;
  float rh[NB], rl[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = cc + 4 * b;
    const float2 v = j < n ? __ldg(r2 + __ldg(dofs + j)) : make_float2(0.f, 0.f);
    rh[b] = v.x;
    rl[b] = v.y;
  }
  float ah[NA], al[NA];
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const float2 f = __ldg(Fp + (a * NB + b) * 32 + lane);
      const float p = __fmul_rn(f.x, rh[b]);
      float e = __fmaf_rn(f.x, rh[b], -p);
      e = __fmaf_rn(f.x, rl[b], e);
      e = __fmaf_rn(f.y, rh[b], e);
      two_sum_acc(hi, lo, p);
      lo = __fadd_rn(lo, e);
    }
    ah[a] = hi;
    al[a] = lo;
  }
#pragma unroll
  for (int a = 0; a < NA; ++a)
#pragma unroll
    for (int o = 8; o <= 16; o <<= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, ah[a], o);
      const float ol = __shfl_xor_sync(0xffffffffu, al[a], o);
      two_sum_acc(ah[a], al[a], oh);
      al[a] = __fadd_rn(al[a], ol);
    }
  if (cc == 0) {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const int row = rr + 8 * a;
      if (row < n) delta[__ldg(pos + s0 + row)] = make_float2(ah[a], al[a]);
    }
  }
}

template <int NB, int NBMAX, typename FT>
__device__ __forceinline__ void apply_dispatch(int nb, int n, int s0, const int* dofs, const FT* Fp,
                                               const double* r, const float2* r2, const int* pos, double* delta,
                                               int lane) {
  if constexpr (NB <= NBMAX) {
    if (nb == NB) {
      if constexpr (std::is_same<FT, float2>::value)
        apply_one_pair<NB>(n, s0, dofs, Fp, r2, pos, reinterpret_cast<float2*>(delta), lane);
      else
        apply_one<NB, FT>(n, s0, dofs, Fp, r, pos, delta, lane);
    } else {
      apply_dispatch<NB + 1, NBMAX, FT>(nb, n, s0, dofs, Fp, r, r2, pos, delta, lane);
    }
  }
}

// Work items w0 <= w < w1 of the work list (one patch per warp), for patches with NBLO <= ceil(n/4)
// <= NBHI.  Warps stride over the range by the number of warps in the grid, so the same kernel runs
// either with one warp per item or as a persistent grid of a few blocks per SM.  Which warp applies a
// patch never changes its arithmetic: every launch shape gives bit-identical corrections.
template <int NBLO, int NBHI, typename FT>
__global__ void __launch_bounds__(256) k_patch_apply(int w0, int w1, const int* __restrict__ work,
                                                     const int* __restrict__ slot_ptr,
                                                     const int* __restrict__ slot_dofs,
                                                     const int64_t* __restrict__ foff,
                                                     const FT* __restrict__ F, const double* __restrict__ r,
                                                     const float2* __restrict__ r2, const int* __restrict__ pos,
                                                     double* __restrict__ delta) {
  pdl_wait();
  const int nwarps = int((int64_t(gridDim.x) * blockDim.x) >> 5);
  const int lane = threadIdx.x & 31;
  for (int w = w0 + int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); w < w1; w += nwarps) {
    const int p = work[w];
    const int s0 = slot_ptr[p], n = slot_ptr[p + 1] - s0;
    apply_dispatch<NBLO, NBHI, FT>((n + 3) >> 2, n, s0, slot_dofs + s0, F + foff[p], r, r2, pos, delta, lane);
  }
}

// ---- symmetric tile layout (FP32 and FP32-pair inverses, patches of at most kSymMaxN DoFs) ----------
// One warp per patch.  Lane l = i + 8 j holds entries (i, j) and (i, j + 4) of every stored tile
// (I, J), I <= J.  With x the local residual:
//   row part:    y_I += T_IJ x_J                 (lane: row i of block I, columns j, j + 4 of block J)
//   column part: y_J += T_IJ^T x_I   (I < J)     (lane: columns j, j + 4 of block J, row i of block I)
// so every stored off-diagonal entry is used twice and the lower triangle is never read.  The row
// partial sums are combined over the four lanes of a row (xor 8, 16), the column partial sums over
// the eight lanes of a column (xor 1, 2, 4); row m of block I is then row part + column part, written
// by the lanes with j == I mod 4.  Fixed order everywhere, so every launch shape gives the same bits.
template <typename FT>
struct SymOps;

template <>
struct SymOps<float> {   // FP32 inverses: FP32 local residual, FP32 products and sums
  using X = float;
  using Vec = float2;    // a lane's two entries of a tile
  struct Acc {
    float v;
  };
  static __device__ __forceinline__ X load_x(const double* r, const float2*, int d) {
    return __double2float_rn(__ldg(r + d));
  }
  static __device__ __forceinline__ X zero_x() { return 0.f; }
  static __device__ __forceinline__ Acc zero() { return Acc{0.f}; }
  static __device__ __forceinline__ void fma_(Acc& a, float e, X x) { a.v = __fmaf_rn(e, x, a.v); }
  static __device__ __forceinline__ void entries(const Vec& v, float& e0, float& e1) {
    e0 = v.x;
    e1 = v.y;
  }
  static __device__ __forceinline__ Acc add(Acc a, Acc b) { return Acc{__fadd_rn(a.v, b.v)}; }
  static __device__ __forceinline__ Acc shfl_xor(Acc a, int o) { return Acc{__shfl_xor_sync(0xffffffffu, a.v, o)}; }
  static __device__ __forceinline__ Acc shfl(Acc a, int src) { return Acc{__shfl_sync(0xffffffffu, a.v, src)}; }
  static __device__ __forceinline__ void store(double* delta, int idx, Acc a) { delta[idx] = double(a.v); }
};

template <>
struct SymOps<float2> {  // FP32-pair inverses: pair products (exact split) with TwoSum accumulation
  using X = float2;
  using Vec = float4;
  struct Acc {
    float hi, lo;
  };
  static __device__ __forceinline__ X load_x(const double*, const float2* r2, int d) { return __ldg(r2 + d); }
  static __device__ __forceinline__ X zero_x() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ Acc zero() { return Acc{0.f, 0.f}; }
  static __device__ __forceinline__ void fma_(Acc& a, float2 e, X x) {
    const float p = __fmul_rn(e.x, x.x);
    float er = __fmaf_rn(e.x, x.x, -p);
    er = __fmaf_rn(e.x, x.y, er);
    er = __fmaf_rn(e.y, x.x, er);
    two_sum_acc(a.hi, a.lo, p);
    a.lo = __fadd_rn(a.lo, er);
  }
  static __device__ __forceinline__ void entries(const Vec& v, float2& e0, float2& e1) {
    e0 = make_float2(v.x, v.y);
    e1 = make_float2(v.z, v.w);
  }
  static __device__ __forceinline__ Acc add(Acc a, Acc b) {
    two_sum_acc(a.hi, a.lo, b.hi);
    a.lo = __fadd_rn(a.lo, b.lo);
    return a;
  }
  static __device__ __forceinline__ Acc shfl_xor(Acc a, int o) {
    return Acc{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
  }
  static __device__ __forceinline__ Acc shfl(Acc a, int src) {
    return Acc{__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src)};
  }
  static __device__ __forceinline__ void store(double* delta, int idx, Acc a) {
    reinterpret_cast<float2*>(delta)[idx] = make_float2(a.hi, a.lo);
  }
};

template <int NT, typename FT>
__device__ __forceinline__ void apply_sym(int n, int s0, const int* __restrict__ dofs, const FT* __restrict__ Fp,
                                          const double* __restrict__ r, const float2* __restrict__ r2,
                                          const int* __restrict__ pos, double* __restrict__ delta, int lane) {
  using O = SymOps<FT>;
  using X = typename O::X;
  using Vec = typename O::Vec;
  using Acc = typename O::Acc;
  using E = FT;
  const int i = lane & 7, j = lane >> 3;
  X xr[NT], xc0[NT], xc1[NT];
#pragma unroll
  for (int I = 0; I < NT; ++I) {
    const int a = 8 * I + i, b0 = 8 * I + j, b1 = b0 + 4;
    xr[I] = a < n ? O::load_x(r, r2, __ldg(dofs + a)) : O::zero_x();
    xc0[I] = b0 < n ? O::load_x(r, r2, __ldg(dofs + b0)) : O::zero_x();
    xc1[I] = b1 < n ? O::load_x(r, r2, __ldg(dofs + b1)) : O::zero_x();
  }
  Acc row[NT], col0[NT], col1[NT];
#pragma unroll
  for (int I = 0; I < NT; ++I) row[I] = col0[I] = col1[I] = O::zero();
  const Vec* T = reinterpret_cast<const Vec*>(Fp) + lane;
#pragma unroll
  for (int I = 0; I < NT; ++I)
#pragma unroll
    for (int J = I; J < NT; ++J) {
      const int t = I * NT - (I * (I - 1)) / 2 + (J - I);   // tiles before row I, then J - I
      E e0, e1;
      O::entries(__ldg(T + 32 * t), e0, e1);
      O::fma_(row[I], e0, xc0[J]);
      O::fma_(row[I], e1, xc1[J]);
      if (I != J) {
        O::fma_(col0[J], e0, xr[I]);
        O::fma_(col1[J], e1, xr[I]);
      }
    }
#pragma unroll
  for (int I = 0; I < NT; ++I) {
    row[I] = O::add(row[I], O::shfl_xor(row[I], 8));
    row[I] = O::add(row[I], O::shfl_xor(row[I], 16));
#pragma unroll
    for (int o = 1; o <= 4; o <<= 1) {
      col0[I] = O::add(col0[I], O::shfl_xor(col0[I], o));
      col1[I] = O::add(col1[I], O::shfl_xor(col1[I], o));
    }
  }
#pragma unroll
  for (int I = 0; I < NT; ++I) {
    const int src = (i & 3) << 3;              // a lane whose column index is i mod 4
    const Acc c0 = O::shfl(col0[I], src), c1 = O::shfl(col1[I], src);
    const Acc y = O::add(row[I], i < 4 ? c0 : c1);
    const int m = 8 * I + i;
    if (j == (I & 3) && m < n) O::store(delta, __ldg(pos + s0 + m), y);
  }
}

template <int NT, int NTMAX, typename FT>
__device__ __forceinline__ void sym_dispatch(int nt, int n, int s0, const int* dofs, const FT* Fp, const double* r,
                                             const float2* r2, const int* pos, double* delta, int lane) {
  if constexpr (NT <= NTMAX) {
    if (nt == NT)
      apply_sym<NT, FT>(n, s0, dofs, Fp, r, r2, pos, delta, lane);
    else
      sym_dispatch<NT + 1, NTMAX, FT>(nt, n, s0, dofs, Fp, r, r2, pos, delta, lane);
  }
}

// Work items w0 <= w < w1 with NTLO <= ceil(n/8) <= NTHI, one warp per patch (or a persistent grid).
template <int NTLO, int NTHI, typename FT>
__global__ void __launch_bounds__(256) k_patch_apply_sym(int w0, int w1, const int* __restrict__ work,
                                                         const int* __restrict__ slot_ptr,
                                                         const int* __restrict__ slot_dofs,
                                                         const int64_t* __restrict__ foff,
                                                         const FT* __restrict__ F, const double* __restrict__ r,
                                                         const float2* __restrict__ r2, const int* __restrict__ pos,
                                                         double* __restrict__ delta) {
  pdl_wait();
  const int nwarps = int((int64_t(gridDim.x) * blockDim.x) >> 5);
  const int lane = threadIdx.x & 31;
  for (int w = w0 + int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); w < w1; w += nwarps) {
    const int p = work[w];
    const int s0 = slot_ptr[p], n = slot_ptr[p + 1] - s0;
    sym_dispatch<NTLO, NTHI, FT>((n + 7) >> 3, n, s0, slot_dofs + s0, F + foff[p], r, r2, pos, delta, lane);
  }
}

// r = rh + rl with rh = fl32(r), rl = fl32(r - rh): the FP32-pair form of a residual, once per DoF.
__global__ void k_split_pairs(const double* __restrict__ r, float2* __restrict__ r2, int n) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = r[i];
  const float h = __double2float_rn(v);
  r2[i] = make_float2(h, __double2float_rn(v - double(h)));
}

template <bool kPairs>
__device__ __forceinline__ void scatter_dof(int i, const int* __restrict__ dptr, const double* __restrict__ weight,
                                            const uint8_t* __restrict__ dir, const double* __restrict__ r,
                                            const double* __restrict__ delta, int mode, double theta, double c1,
                                            double c2, double* __restrict__ zout, double* __restrict__ d,
                                            double* __restrict__ x) {
  double z;
  if (dir[i]) {
    z = r[i];
  } else if (kPairs) {
    // corrections are FP32 pairs: sum them in pair arithmetic, convert once
    const float2* d2 = reinterpret_cast<const float2*>(delta);
    float hi = 0.f, lo = 0.f;
    for (int e = dptr[i]; e < dptr[i + 1]; ++e) {
      const float2 v = d2[e];
      two_sum_acc(hi, lo, v.x);
      lo = __fadd_rn(lo, v.y);
    }
    z = double(hi) + double(lo);
    if (weight) z *= weight[i];
  } else {
    z = 0.0;
    const int e0 = dptr[i], e1 = dptr[i + 1];
    if (weight) {
      const double wi = weight[i];
      for (int e = e0; e < e1; ++e) z = __dadd_rn(z, __dmul_rn(delta[e], wi));
    } else {
      for (int e = e0; e < e1; ++e) z += delta[e];
    }
  }
  switch (mode) {
    case 0:
      zout[i] = z;
      break;
    case 1: {
      const double dn = z / theta;
      d[i] = dn;
      x[i] = dn;
      break;
    }
    case 2: {
      const double dn = z / theta;
      d[i] = dn;
      x[i] = x[i] + dn;
      break;
    }
    default: {
      const double dn = __dadd_rn(__dmul_rn(c1, d[i]), __dmul_rn(c2, z));
      d[i] = dn;
      x[i] = x[i] + dn;
      break;
    }
  }
}

template <bool kPairs>
__global__ void __launch_bounds__(256) k_vanka_scatter(int ndof, const int* __restrict__ dptr,
                                                       const double* __restrict__ weight,
                                                       const uint8_t* __restrict__ dir,
                                                       const double* __restrict__ r,
                                                       const double* __restrict__ delta, int mode,
                                                       double theta, double c1, double c2,
                                                       double* __restrict__ zout, double* __restrict__ d,
                                                       double* __restrict__ x) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ndof) return;
  scatter_dof<kPairs>(i, dptr, weight, dir, r, delta, mode, theta, c1, c2, zout, d, x);
}

// ---- group forms (one launch over the members of a group solve) ---------------------------------
template <bool kPairs>
__global__ void __launch_bounds__(256) k_group_scatter(const __grid_constant__ GroupScatterArgs a) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= a.prefix[a.count]) return;
  const int m = group_member(a.prefix, a.count, gi);
  const GroupPatch& P = a.P[m];
  scatter_dof<kPairs>(gi - a.prefix[m], P.dof_ptr, P.weight, P.dir, a.r[m], a.delta[m], a.mode, a.theta[m], a.c1[m],
                      a.c2[m], a.z[m], a.d[m], a.x[m]);
}

__global__ void k_group_split_pairs(const __grid_constant__ GroupApplyArgs a) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= a.dprefix[a.count]) return;
  const int m = group_member(a.dprefix, a.count, gi), i = gi - a.dprefix[m];
  const double v = a.r[m][i];
  const float h = __double2float_rn(v);
  a.r2[m][i] = make_float2(h, __double2float_rn(v - double(h)));
}

// One warp per patch of any member, in each member's own work order and storage layout.
template <int NBMAX, typename FT>
__global__ void __launch_bounds__(256) k_group_apply(const __grid_constant__ GroupApplyArgs a) {
  const int gw = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  if (gw >= a.prefix[a.count]) return;
  const int m = group_member(a.prefix, a.count, gw);
  const GroupPatch& P = a.P[m];
  const int lane = threadIdx.x & 31;
  const int p = P.work[gw - a.prefix[m]];
  const int s0 = P.slot_ptr[p], n = P.slot_ptr[p + 1] - s0;
  const FT* F = static_cast<const FT*>(P.factors) + P.foff[p];
  if constexpr (!std::is_same<FT, double>::value) {
    if (P.sym) {
      sym_dispatch<1, 10, FT>((n + 7) >> 3, n, s0, P.slot_dofs + s0, F, a.r[m], a.r2[m], P.slot_pos, a.delta[m], lane);
      return;
    }
  }
  apply_dispatch<1, NBMAX, FT>((n + 3) >> 2, n, s0, P.slot_dofs + s0, F, a.r[m], a.r2[m], P.slot_pos, a.delta[m],
                               lane);
}

// Blocks of one launch over `items` work items: one warp per item, or (per_sm > 0) at most per_sm
// blocks per SM with the warps striding over the items.
int apply_blocks(int items, const ApplySched& sc, int nsm) {
  const int warps = sc.threads / 32;
  int blocks = (items + warps - 1) / warps;
  if (sc.per_sm > 0) blocks = std::min(blocks, sc.per_sm * std::max(nsm, 1));
  return std::max(blocks, 1);
}

template <int NBLO, int NBHI, typename FT>
int launch_range(const Patches& P, const ApplySched& sc, int w0, int w1, const double* r, const float2* r2,
                 double* delta, cudaStream_t s) {
  if (w1 <= w0) return 0;
  launch(k_patch_apply<NBLO, NBHI, FT>, dim3(apply_blocks(w1 - w0, sc, P.nsm)), dim3(sc.threads), 0, s, 
      w0, w1, P.work, P.slot_ptr, P.slot_dofs, P.foff, static_cast<const FT*>(P.factors), r, r2, P.slot_pos, delta);
  return 1;
}

template <int NTLO, int NTHI, typename FT>
int launch_range_sym(const Patches& P, const ApplySched& sc, int w0, int w1, const double* r, const float2* r2,
                     double* delta, cudaStream_t s) {
  if (w1 <= w0) return 0;
  launch(k_patch_apply_sym<NTLO, NTHI, FT>, dim3(apply_blocks(w1 - w0, sc, P.nsm)), dim3(sc.threads), 0, s, 
      w0, w1, P.work, P.slot_ptr, P.slot_dofs, P.foff, static_cast<const FT*>(P.factors), r, r2, P.slot_pos, delta);
  return 1;
}

// Symmetric layout: the same launch shapes; the size classes of ceil(n/4) map to ceil(n/8) ranges
// 1-2, 3-5, 6-10 and 10 (n <= kSymMaxN = 80).
template <typename FT>
int apply_sym_prec(const Patches& P, const ApplySched& sc, const double* r, const float2* r2, double* delta,
                   cudaStream_t s) {
  if (!sc.split) {
    if (P.nb_max <= 10) return launch_range_sym<1, 5, FT>(P, sc, 0, P.npatch, r, r2, delta, s);
    return launch_range_sym<1, 10, FT>(P, sc, 0, P.npatch, r, r2, delta, s);
  }
  int k = 0;
  k += launch_range_sym<10, 10, FT>(P, sc, P.cls_lo[3], P.cls_hi[3], r, r2, delta, s);
  k += launch_range_sym<6, 10, FT>(P, sc, P.cls_lo[2], P.cls_hi[2], r, r2, delta, s);
  k += launch_range_sym<3, 5, FT>(P, sc, P.cls_lo[1], P.cls_hi[1], r, r2, delta, s);
  k += launch_range_sym<1, 2, FT>(P, sc, P.cls_lo[0], P.cls_hi[0], r, r2, delta, s);
  return k;
}

template <typename FT>
int apply_prec(const Patches& P, const ApplySched& sc, const double* r, const float2* r2, double* delta,
               cudaStream_t s) {
  if (!sc.split) {
    // one launch over every patch of the level; the per-warp dispatch covers all sizes
    if (P.nb_max <= 10) return launch_range<1, 10, FT>(P, sc, 0, P.npatch, r, r2, delta, s);
    if (P.nb_max <= 19) return launch_range<1, 19, FT>(P, sc, 0, P.npatch, r, r2, delta, s);
    if (P.nb_max <= 32) return launch_range<1, 32, FT>(P, sc, 0, P.npatch, r, r2, delta, s);
    return launch_range<1, 42, FT>(P, sc, 0, P.npatch, r, r2, delta, s);
  }
  // one launch per size class, each compiled for its own range of sizes (fewer registers, so more
  // resident warps, for the small classes)
  int k = 0;
  k += launch_range<33, 42, FT>(P, sc, P.cls_lo[4], P.cls_hi[4], r, r2, delta, s);
  k += launch_range<20, 32, FT>(P, sc, P.cls_lo[3], P.cls_hi[3], r, r2, delta, s);
  k += launch_range<11, 19, FT>(P, sc, P.cls_lo[2], P.cls_hi[2], r, r2, delta, s);
  k += launch_range<5, 10, FT>(P, sc, P.cls_lo[1], P.cls_hi[1], r, r2, delta, s);
  k += launch_range<1, 4, FT>(P, sc, P.cls_lo[0], P.cls_hi[0], r, r2, delta, s);
  return k;
}

}  // namespace

namespace {

template <typename FT>
void launch_factor(const Csr& A, const PatchElems* elems, const Patches& P, void* factors, int* status, size_t smem,
                   int smem_cap, cudaStream_t s) {
  if (elems) {
    cudaFuncSetAttribute(k_patch_factor<FT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_cap);
    k_patch_factor<FT, true><<<P.npatch, kFactorThreads, smem, s>>>(A, *elems, P.slot_ptr, P.slot_dofs, P.foff,
                                                                     static_cast<FT*>(factors), status, P.sym);
  } else {
    cudaFuncSetAttribute(k_patch_factor<FT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_cap);
    k_patch_factor<FT, false><<<P.npatch, kFactorThreads, smem, s>>>(A, PatchElems{}, P.slot_ptr, P.slot_dofs,
                                                                      P.foff, static_cast<FT*>(factors), status,
                                                                      P.sym);
  }
}

}  // namespace

int patch_factor(const Csr& A, const Patches& P, int prec, void* factors, int* status, cudaStream_t s,
                 const PatchElems* elems) {
  if (P.npatch == 0) return 0;
  // shared bytes n*n*8 + n*12 for the largest patch of the level (n <= 4 * nb_max <= kMaxPatch: 168
  // FP64 rows of 168 are 226 KB, within the 227 KB a block may use).  The function attribute is always
  // set to the bound for n = kMaxPatch (the same value from every thread, so concurrent setups cannot
  // lower it under each other's launches).
  const int nmax = 4 * P.nb_max;
  const size_t smem = size_t(nmax) * nmax * 8 + size_t(nmax) * 12;
  const int smem_cap = kMaxPatch * kMaxPatch * 8 + kMaxPatch * 12;
  if (nmax > kMaxPatch) return -1;   // the caller reports VK_ERR_ARG: nothing is left unfactored silently
  if (prec == 0)
    launch_factor<double>(A, elems, P, factors, status, smem, smem_cap, s);
  else if (prec == 1)
    launch_factor<float>(A, elems, P, factors, status, smem, smem_cap, s);
  else
    launch_factor<float2>(A, elems, P, factors, status, smem, smem_cap, s);
  return 1;
}

int patch_apply_sched(const Patches& P, const ApplySched& sc, const double* r, float2* r2, double* delta,
                      cudaStream_t s) {
  if (P.npatch == 0) return 0;
  if (P.prec == 0) return apply_prec<double>(P, sc, r, nullptr, delta, s);
  if (P.prec == 1)
    return P.sym ? apply_sym_prec<float>(P, sc, r, nullptr, delta, s) : apply_prec<float>(P, sc, r, nullptr, delta, s);
  // FP32-pair inverses: split the residual once per DoF first
  const int n = P.ndof;
  launch(k_split_pairs, dim3((n + 255) / 256), dim3(256), 0, s, r, r2, n);
  return 1 + (P.sym ? apply_sym_prec<float2>(P, sc, r, r2, delta, s) : apply_prec<float2>(P, sc, r, r2, delta, s));
}

int patch_apply(const Patches& P, const double* r, float2* r2, double* delta, cudaStream_t s) {
  return patch_apply_sched(P, P.sched, r, r2, delta, s);
}

template <typename FT>
int group_apply_prec(const GroupApplyArgs& a, cudaStream_t s) {
  const int blocks = (a.prefix[a.count] + 7) / 8;   // 8 warps of 256 threads
  if (a.nb_max <= 10)
    k_group_apply<10, FT><<<blocks, 256, 0, s>>>(a);
  else if (a.nb_max <= 19)
    k_group_apply<19, FT><<<blocks, 256, 0, s>>>(a);
  else if (a.nb_max <= 32)
    k_group_apply<32, FT><<<blocks, 256, 0, s>>>(a);
  else
    k_group_apply<42, FT><<<blocks, 256, 0, s>>>(a);
  return 1;
}

int group_patch_apply(const GroupApplyArgs& a, cudaStream_t s) {
  if (a.count == 0 || a.prefix[a.count] == 0) return 0;
  if (a.prec == 0) return group_apply_prec<double>(a, s);
  if (a.prec == 1) return group_apply_prec<float>(a, s);
  k_group_split_pairs<<<(a.dprefix[a.count] + 255) / 256, 256, 0, s>>>(a);
  return 1 + group_apply_prec<float2>(a, s);
}

int group_vanka_scatter(const GroupScatterArgs& a, cudaStream_t s) {
  if (a.count == 0 || a.prefix[a.count] == 0) return 0;
  const int blocks = (a.prefix[a.count] + 255) / 256;
  if (a.prec == 2)
    k_group_scatter<true><<<blocks, 256, 0, s>>>(a);
  else
    k_group_scatter<false><<<blocks, 256, 0, s>>>(a);
  return 1;
}

int vanka_scatter(const Patches& P, int ndof, const uint8_t* dir, const double* r, const double* delta,
                   int mode, double theta, double c1, double c2, double* out_z, double* d, double* x,
                   cudaStream_t s) {
  if (P.prec == 2)
    launch(k_vanka_scatter<true>, dim3((ndof + 255) / 256), dim3(256), 0, s, ndof, P.dof_ptr, P.weight, dir, r, delta, mode,
                                                             theta, c1, c2, out_z, d, x);
  else
    launch(k_vanka_scatter<false>, dim3((ndof + 255) / 256), dim3(256), 0, s, ndof, P.dof_ptr, P.weight, dir, r, delta, mode,
                                                              theta, c1, c2, out_z, d, x);
  return 1;
}

}  // namespace gpu
}  // namespace vk
