// Tensor-core patch solves of vk_solve_batch on the 5th-generation tensor cores (tcgen05, TMEM, TMA).
//
// Algorithm 1's patch solve for 16 right-hand sides at once is the dense contraction
// delta_i[n x 16] = A_i^{-1}[n x n] R_i[n x 16].  One tcgen05.mma (M = 128, K = 16, BF16 or FP16
// inputs, FP32 accumulator in tensor memory) takes G patches stacked along M: patch j of a group owns
// rows [8 MB j, 8 MB j + n_j) of the A tile and columns [16 j, 16 j + 16) of the B tile, so the
// accumulator block (j, j) is its result and the off-diagonal blocks are ignored.  Classes by patch
// size: n <= 40 -> 3 patches of 40 rows (N = 48); n <= 64 -> 2 of 64 (N = 32); n <= 128 -> 1 (N = 16).
//
// Per CTA (128 threads, persistent over the groups of one class, software-pipelined):
//   * the scaled inverses are stored in HBM as 8x8 core matrices (128 bytes: 8 rows of 8 16-bit
//     values), only ceil(n/8)^2 of them per patch, and copied into shared memory by one thread with
//     cp.async.bulk (TMA, completion counted in bytes on an mbarrier), double-buffered: the copies
//     of group g + grid are issued right after the MMAs of group g;
//   * every thread holds 4 right-hand sides of up to 5 residual rows of the group in registers,
//     loaded one iteration ahead (their DoF indices two iterations ahead) from per-group tables
//     built at setup, so the gathers of the next group are in flight during this group's MMAs and
//     epilogue; the rows are scaled per column by the column's largest magnitude over the patch (a
//     column's result does not depend on the other columns), rounded to 16 bits and stored as the
//     B tile in core-matrix order;
//   * one thread issues the K/16 MMAs and commits them to an mbarrier;
//   * warp w reads accumulator lanes 32w..32w+31 (row 32w + lane) with tcgen05.ld and writes the
//     unscaled corrections of its patch row to delta[slot][16] (the layout k_scatter_mm sums).
// Shared-memory operand layout (no swizzle, K-major): core matrix (row block m, K chunk c) of the A
// tile at (c/2) * 4096 + (c%2) * 2048 + 128 m, so the K-adjacent core matrix is 2048 bytes away
// (leading byte offset) and the next row block 128 bytes (stride byte offset); B likewise with N/8
// row blocks (the results of the GPU tests confirm this reading of the two offsets).  Every mbarrier
// wait is bounded (about 2 s of %globaltimer); on expiry the CTA records
// VK_ERR_TIMEOUT in *err, waits (bounded) for its MMAs in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

#include "gpu.h"

namespace vk {
namespace gpu {

namespace {

constexpr int kNR = 16;
constexpr int kTcThreads = 128;
constexpr uint64_t kWaitNs = 2000000000ull;   // bound of every mbarrier wait
constexpr int kErrTimeout = 6;                 // VK_ERR_TIMEOUT

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > kWaitNs) return false;
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, 16-bit inputs, FP32 accumulate
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading / stride byte offsets (16-byte units),
// fixed 0b001 at bits 46-48, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t((lbo & 0x3FFFFu) >> 4) << 16) |
         (uint64_t((sbo & 0x3FFFFu) >> 4) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B both BF16 or both FP16, K-major,
// N / 8 at bits 17-22, M / 16 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool half) {
  return (1u << 4) | ((half ? 0u : 1u) << 7) | ((half ? 0u : 1u) << 10) | (uint32_t(N >> 3) << 17) |
         (uint32_t(M >> 4) << 24);
}

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

template <int MB, int G, int KS>
struct TcShape {
  static constexpr int R = 8 * MB;                 // A rows per patch slot
  static constexpr int N = 16 * G;                 // MMA N
  static constexpr int K = 16 * KS;                // padded K
  static constexpr int TCOLS = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
  static constexpr int A_KH = 16 * 128;            // K-adjacent core matrices of A (128 rows)
  static constexpr int A_KS = 2 * A_KH;            // one K-step of A
  static constexpr int A_STAGE = KS * A_KS;
  static constexpr int B_KH = (N / 8) * 128;       // K-adjacent core matrices of B
  static constexpr int B_KS = 2 * B_KH;
  static constexpr int B_BYTES = KS * B_KS;
  static constexpr int QN = G * K * 4;             // float4 items (row k of slot j, 4 right-hand sides)
  static constexpr int QI = (QN + kTcThreads - 1) / kTcThreads;
  // shared bytes: 2 A stages, B, 2 x column maxima, 3 mbarriers + TMEM address
  static constexpr int SMEM = 2 * A_STAGE + B_BYTES + 2 * 4 * G * kNR + 64;
  static_assert(G * R <= 128, "patch slots exceed the 128 accumulator lanes");
  static_assert(N % 16 == 0 && N >= 16 && N <= 256, "M = 128 needs N a multiple of 16 in 16..256");
  static_assert((K * 4) % 32 == 0 && QN % 32 == 0, "a warp's items must share one patch slot");
};

// One size class: group g holds the work items lo + G g .. lo + G g + G - 1.
//   gdof[(g G + j) K + k]  DoF of row k of slot j (-1 past the patch or for an empty slot)
//   gpos[g 128 + t]        delta row of accumulator lane t = 8 MB j + r (-1: no patch row)
//   gslot[g G + j]         (byte offset of the core matrices: low, high word; n; patch id), n = 0: empty
template <int MB, int G, int KS, bool kHalf>
__global__ void __launch_bounds__(kTcThreads, 6) k_patch_tc(TcClass C, const uint8_t* __restrict__ frag,
                                                         const float* __restrict__ ascale,
                                                         const float* __restrict__ rhs, float* __restrict__ delta,
                                                         int* __restrict__ err) {
  using S = TcShape<MB, G, KS>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Abuf = smem;                                           // [2][A_STAGE]
  uint8_t* Bt = smem + 2 * S::A_STAGE;                            // [B_BYTES]
  int* cmax = reinterpret_cast<int*>(Bt + S::B_BYTES);            // [2][G][16] float bits (>= 0)
  uint64_t* bars = reinterpret_cast<uint64_t*>(cmax + 2 * G * kNR);  // abar[0], abar[1], dbar
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 3);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ng = C.ngroups, grid = int(gridDim.x);
  // zero both A stages once: K chunks a patch does not fill keep finite values (zeros or an
  // earlier patch's entries), which the zero rows of its B block cancel
  for (int i = tid; i < 2 * S::A_STAGE / 16; i += kTcThreads) reinterpret_cast<uint4*>(Abuf)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < 2 * G * kNR; i += kTcThreads) cmax[i] = 0;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, S::TCOLS);
    tmem_relinquish();
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // ---- pipeline helpers -------------------------------------------------------------------------
  auto load_meta = [&](int g, int4 (&m)[G]) {
#pragma unroll
    for (int j = 0; j < G; ++j) m[j] = g < ng ? __ldg(C.gslot + int64_t(g) * G + j) : make_int4(0, 0, 0, 0);
  };
  // thread 0: start the copies of a group's inverses into stage b
  auto issue = [&](int b, const int4 (&m)[G]) {
    uint32_t bytes = 0;
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const int nb = (m[j].z + 7) >> 3;
      bytes += uint32_t(nb * nb * 128);
    }
    mbar_expect_tx(&bars[b], bytes);
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const int nb = (m[j].z + 7) >> 3;
      const uint8_t* src = frag + ((int64_t(uint32_t(m[j].y)) << 32) | uint32_t(m[j].x));
      for (int c = 0; c < nb; ++c)
        bulk_g2s(Abuf + b * S::A_STAGE + (c >> 1) * S::A_KS + (c & 1) * S::A_KH + (MB * j) * 128,
                 src + int64_t(c) * nb * 128, uint32_t(nb * 128), &bars[b]);
    }
  };
  auto load_idx = [&](int g, int (&idx)[S::QI]) {
#pragma unroll
    for (int i = 0; i < S::QI; ++i) {
      const int q = tid + kTcThreads * i;
      idx[i] = (g < ng && q < S::QN) ? __ldg(C.gdof + int64_t(g) * G * S::K + (q >> 2)) : -1;
    }
  };
  auto load_rhs = [&](const int (&idx)[S::QI], float4 (&v)[S::QI]) {
#pragma unroll
    for (int i = 0; i < S::QI; ++i) {
      const int q = tid + kTcThreads * i;
      v[i] = idx[i] >= 0 ? __ldg(reinterpret_cast<const float4*>(rhs + int64_t(idx[i]) * kNR) + (q & 3))
                         : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };

  uint32_t aphase[2] = {0, 0}, dphase = 0;
  bool ok = true;
  // thread 0's record of its asynchronous work in flight: copies per stage, MMAs
  bool copy_pending[2] = {false, false}, mma_pending = false;
  int4 meta_next[G];
  float4 cur[S::QI];
  int nidx[S::QI];
  {
    const int g0 = blockIdx.x;
    if (tid == 0) {
      int4 m0[G];
      load_meta(g0, m0);
      if (g0 < ng) {
        issue(0, m0);
        copy_pending[0] = true;
      }
      load_meta(g0 + grid, meta_next);
    }
    int idx0[S::QI];
    load_idx(g0, idx0);
    load_rhs(idx0, cur);
    load_idx(g0 + grid, nidx);
  }
  int it = 0;
  for (int g = blockIdx.x; g < ng; g += grid, ++it) {
    const int b = it & 1;
    int* cb = cmax + b * G * kNR;
    // ---- 1. column maxima of the group's residual block: warp maxima over its 8 rows, then smem --
#pragma unroll
    for (int i = 0; i < S::QI; ++i) {
      const int q0 = kTcThreads * i + warp * 32;        // first item of this warp (warp-uniform)
      if (q0 < S::QN) {
        const int q = q0 + lane;
        float m[4] = {fabsf(cur[i].x), fabsf(cur[i].y), fabsf(cur[i].z), fabsf(cur[i].w)};
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
          for (int o = 4; o < 32; o <<= 1) m[e] = fmaxf(m[e], __shfl_xor_sync(0xffffffffu, m[e], o));
        if (lane < 4) {
          const int j = q / (S::K * 4);
#pragma unroll
          for (int e = 0; e < 4; ++e) atomicMax(cb + j * kNR + 4 * lane + e, __float_as_int(m[e]));
        }
      }
    }
    __syncthreads();
    // ---- 2. scale each column, round to 16 bits, B tile in K-major core-matrix order --------------
    //      element (n = 16 j + c, k) at (k/16) B_KS + ((k/8)%2) B_KH + (n/8) 128 + (n%8) 16 + (k%8) 2
#pragma unroll
    for (int i = 0; i < S::QI; ++i) {
      const int q = tid + kTcThreads * i;
      if (q < S::QN) {
        const int j = q / (S::K * 4), k = (q >> 2) % S::K, c4 = q & 3;
        const float v[4] = {cur[i].x, cur[i].y, cur[i].z, cur[i].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int n = 16 * j + 4 * c4 + e;
          const float mx = __int_as_float(cb[j * kNR + 4 * c4 + e]);
          const float x = mx > 0.f ? v[e] * (1.f / mx) : 0.f;
          const int off = (k >> 4) * S::B_KS + ((k >> 3) & 1) * S::B_KH + (n >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
          if constexpr (kHalf)
            *reinterpret_cast<__half*>(Bt + off) = __float2half_rn(x);
          else
            *reinterpret_cast<__nv_bfloat16*>(Bt + off) = __float2bfloat16_rn(x);
        }
      }
    }
    fence_proxy_async();
    __syncthreads();
    // ---- 3. MMAs (thread 0), then the next group's copies into the other stage -------------------
    if (tid == 0) {
      if (mbar_wait(&bars[b], aphase[b])) {
        copy_pending[b] = false;
        aphase[b] ^= 1u;
      } else {
        atomicExch(err, kErrTimeout);
        ok = false;
      }
      if (ok) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(Abuf + b * S::A_STAGE), b0 = smem_u32(Bt);
        constexpr uint32_t idesc = idesc_f16(128, S::N, kHalf);
#pragma unroll
        for (int kk = 0; kk < KS; ++kk)
          tc_mma(tmem, sdesc(a0 + kk * S::A_KS, S::A_KH, 128), sdesc(b0 + kk * S::B_KS, S::B_KH, 128), idesc,
                 kk > 0 ? 1u : 0u);
        tc_commit(&bars[2]);
        mma_pending = true;
        // stage b ^ 1 was read by the previous group's MMAs, which completed before its epilogue
        if (g + grid < ng) {
          issue(b ^ 1, meta_next);
          copy_pending[b ^ 1] = true;
        }
        load_meta(g + 2 * grid, meta_next);
      }
    }
    // ---- 4. the next group's residual rows and the group after that's DoF indices (in flight
    //         during this group's MMAs and epilogue) -------------------------------------------------
    load_rhs(nidx, cur);
    load_idx(g + 2 * grid, nidx);
    const int t = 32 * warp + lane;
    const int prow = __ldg(C.gpos + int64_t(g) * 128 + t);
    const int jt = t / S::R < G ? t / S::R : 0;
    const float sa = prow >= 0 ? __ldg(ascale + __ldg(C.gslot + int64_t(g) * G + jt).w) : 0.f;
    // every thread learns whether the MMAs were issued (a timed-out copy skips them)
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok) break;
    if (mbar_wait(&bars[2], dphase)) {
      if (tid == 0) mma_pending = false;
      dphase ^= 1u;
    } else {
      atomicExch(err, kErrTimeout);
      ok = false;
    }
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok) break;
    tc_fence_after();
    // ---- 5. epilogue: accumulator lane t -> slot jt, row t - R jt ----------------------------------
    float acc[G][16];
#pragma unroll
    for (int j = 0; j < G; ++j) tc_ld16(tmem + (uint32_t(32 * warp) << 16) + uint32_t(16 * j), acc[j]);
    tc_wait_ld();
    if (prow >= 0) {
      float* o = delta + int64_t(prow) * kNR;
#pragma unroll
      for (int jj = 0; jj < G; ++jj)
        if (jj == jt) {
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            float4 v;
            v.x = acc[jj][4 * c4 + 0] * (sa * __int_as_float(cb[jj * kNR + 4 * c4 + 0]));
            v.y = acc[jj][4 * c4 + 1] * (sa * __int_as_float(cb[jj * kNR + 4 * c4 + 1]));
            v.z = acc[jj][4 * c4 + 2] * (sa * __int_as_float(cb[jj * kNR + 4 * c4 + 2]));
            v.w = acc[jj][4 * c4 + 3] * (sa * __int_as_float(cb[jj * kNR + 4 * c4 + 3]));
            reinterpret_cast<float4*>(o)[c4] = v;
          }
        }
    }
    // the other column-maxima buffer starts from zero for the next group
    for (int i = tid; i < G * kNR; i += kTcThreads) cmax[(b ^ 1) * G * kNR + i] = 0;
    tc_fence_before();
    __syncthreads();
  }
  if (tid == 0) {
    // after a timeout: give the copies and MMAs still in flight a bounded chance to land before the
    // shared and tensor memory they target is released (nothing is pending after a normal loop end)
    if (mma_pending) mbar_wait(&bars[2], dphase);
    for (int b = 0; b < 2; ++b)
      if (copy_pending[b]) mbar_wait(&bars[b], aphase[b]);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, S::TCOLS);
}

// Pack the FP64 warp-packed inverse of each patch (kernels_patch.cu layout) into 8x8 core matrices
// of 16-bit values scaled by 1 / ascale[p] (ascale computed by the fragment packer): chunk c of K,
// row block m at byte (c * nb + m) * 128, row r8 at + 16 r8, column k8 at + 2 k8, nb = ceil(n/8).
template <bool kHalf>
__global__ void k_pack_tc(const int* __restrict__ slot_ptr, const int64_t* __restrict__ foff64,
                          const double* __restrict__ inv64, const float* __restrict__ ascale,
                          const int64_t* __restrict__ foff_tc, uint8_t* __restrict__ frag) {
  const int p = blockIdx.x;
  const int n = slot_ptr[p + 1] - slot_ptr[p];
  const int NB4 = (n + 3) / 4, nb = (n + 7) / 8;
  const double* src = inv64 + foff64[p];
  const double inv = 1.0 / double(ascale[p]);
  uint32_t* dst = reinterpret_cast<uint32_t*>(frag + foff_tc[p]);
  // one 32-bit word = two adjacent columns of a row
  for (int e = threadIdx.x; e < nb * nb * 32; e += blockDim.x) {
    const int cm = e >> 5, w = e & 31;
    const int c = cm / nb, m = cm - c * nb;
    const int row = 8 * m + (w >> 2), col = 8 * c + 2 * (w & 3);
    auto at = [&](int rr, int cc) -> double {
      if (rr >= n || cc >= n) return 0.0;
      return src[((rr >> 3) * NB4 + (cc >> 2)) * 32 + (rr & 7) + 8 * (cc & 3)];
    };
    dst[e] = pack2<kHalf>(float(at(row, col) * inv), float(at(row, col + 1) * inv));
  }
}

template <int MB, int G, int KS, bool kHalf>
int launch_tc(const TcPatches& T, int c, const float* rhs, float* delta, int* err, cudaStream_t s) {
  using S = TcShape<MB, G, KS>;
  const TcClass& C = T.cls[c];
  if (C.ngroups <= 0) return 0;
  static_assert(S::SMEM <= 227 * 1024, "shared memory");
  auto kern = k_patch_tc<MB, G, KS, kHalf>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  // resident CTAs per SM, from the kernel's registers and shared memory (228 KB per SM, 1 KB of it
  // reserved per CTA), 2048 threads, and the 512 tensor-memory columns
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, kern);
  const int regs = fa.numRegs > 0 ? (fa.numRegs + 7) / 8 * 8 : 64;
  int occ = 65536 / (regs * kTcThreads);
  occ = std::min(occ, (228 * 1024) / (S::SMEM + int(fa.sharedSizeBytes) + 1024));
  occ = std::min(occ, 2048 / kTcThreads);
  occ = std::min(occ, 512 / S::TCOLS);
  occ = std::max(occ, 1);
  const int grid = C.ngroups < occ * T.nsm ? C.ngroups : occ * T.nsm;
  kern<<<grid, kTcThreads, S::SMEM, s>>>(C, T.frag, T.ascale, rhs, delta, err);
  return 1;
}

}  // namespace

int pack_tc(const Patches& P, const double* inv64, const float* ascale, const int64_t* foff_tc, void* frag, bool half,
            cudaStream_t s) {
  if (P.npatch == 0) return 0;
  if (half)
    k_pack_tc<true><<<P.npatch, 128, 0, s>>>(P.slot_ptr, P.foff, inv64, ascale, foff_tc, static_cast<uint8_t*>(frag));
  else
    k_pack_tc<false><<<P.npatch, 128, 0, s>>>(P.slot_ptr, P.foff, inv64, ascale, foff_tc,
                                              static_cast<uint8_t*>(frag));
  return 1;
}

int patch_apply_tc(const TcPatches& T, bool half, const float* rhs, float* delta, int* err, cudaStream_t s) {
  int k = 0;
  if (half) {
    k += launch_tc<16, 1, 8, true>(T, 2, rhs, delta, err, s);
    k += launch_tc<8, 2, 4, true>(T, 1, rhs, delta, err, s);
    k += launch_tc<5, 3, 3, true>(T, 0, rhs, delta, err, s);
  } else {
    k += launch_tc<16, 1, 8, false>(T, 2, rhs, delta, err, s);
    k += launch_tc<8, 2, 4, false>(T, 1, rhs, delta, err, s);
    k += launch_tc<5, 3, 3, false>(T, 0, rhs, delta, err, s);
  }
  return k;
}

}  // namespace gpu
}  // namespace vk
