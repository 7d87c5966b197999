// Tensor-core patch solves of vk_solve_batch on the 5th-generation tensor cores (tcgen05, TMEM, TMA).
//
// Algorithm 1's patch solve for 16 right-hand sides at once is the dense contraction
// delta_i[n x 16] = A_i^{-1}[n x n] R_i[n x 16].  One tcgen05.mma (M = 128, K = 16, BF16 or FP16
// inputs, FP32 accumulator in tensor memory) takes G patches stacked along M: patch j of a group owns
// rows [8 MB j, 8 MB j + n_j) of the A tile and columns [16 j, 16 j + 16) of the B tile, so the
// accumulator block (j, j) is its result and the off-diagonal blocks are ignored.  Classes by patch
// size: n <= 40 -> 3 patches of 40 rows (N = 48); n <= 64 -> 2 of 64 (N = 32); n <= 128 -> 1 (N = 16).
//
// Per CTA (persistent over the groups of one class; 9 warps in three roles joined by mbarriers):
//   * producer (one thread): a group's scaled inverses are stored in HBM as the exact image of the
//     MMA's A operand in shared memory (8x8 core matrices of 128 bytes, K chunk after K chunk, only
//     the chunks its largest patch needs: 10 KB for three 39-DoF patches); it copies each image into
//     a 3-stage shared-memory ring with one cp.async.bulk (TMA, completion counted in bytes on an
//     mbarrier), then issues the K/16 MMAs of a group into one of two tensor-memory accumulators and
//     commits them to the barriers that free the A stage, the B stage and fill the accumulator;
//   * gather (warps 4-7): every thread holds 4 right-hand sides of up to 5 residual rows of a group
//     in registers, loaded one group ahead (their DoF indices two groups ahead) from per-group tables
//     built at setup; with FP16 the rows are scaled per column by the column's largest magnitude over
//     the patch (FP16's exponent range; BF16 rounds them unscaled), rounded to 16 bits and stored as
//     the B tile in core-matrix order (2 stages); a column's result never depends on the others;
//   * read-back (warps 0-3): warp w reads accumulator lanes 32w..32w+31 (row 32w + lane) with
//     tcgen05.ld, releases the accumulator and writes the unscaled corrections of its patch row to
//     delta[slot][16] (the layout k_scatter_mm sums).
// Shared-memory operand layout (no swizzle, K-major): core matrix (row block m, K chunk c) of the A
// tile at (c/2) * 4096 + (c%2) * 2048 + 128 m, so the K-adjacent core matrix is 2048 bytes away
// (leading byte offset) and the next row block 128 bytes (stride byte offset); B likewise with N/8
// row blocks (the results of the GPU tests confirm this reading of the two offsets).  Every mbarrier
// wait is bounded (about 2 s of %globaltimer); on expiry the CTA records VK_ERR_TIMEOUT in *err and
// raises a shared abort flag that ends the other roles' waits, the producer waits (bounded) for its
// copies and MMAs still in flight, and the tensor memory is freed before the CTA returns.  (A test
// exercises this path by announcing one group's copy without issuing it: skip_group.)
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

#include "gpu.h"

namespace vk {
namespace gpu {

namespace {

constexpr int kNR = 16;
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

// One potentially blocking test: the thread may be suspended (up to the hint, 0.1 ms) until the
// phase completes, instead of spinning on the barrier.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
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

// Roles of the 288 threads of a CTA: warps 0-3 read the accumulators back (warp w owns tensor-memory
// lanes 32w..32w+31), warps 4-7 build the B tiles, lane 0 of warp 8 issues the bulk copies and the
// MMAs.  The roles hand groups to each other through mbarriers only (no block-wide barrier inside the
// loop), so the gather of one group, the copies and MMAs of the next ones and the read-back of the
// previous one overlap.
constexpr int kTcWarps = 9, kTcThreadsWs = 32 * kTcWarps;
constexpr int kSA = 3;   // A stages (bulk-copy ring)
constexpr int kSB = 2;   // B stages
constexpr int kSC = 4;   // column-maximum slots (2 kSB: see the epilogue)

template <int MB, int G, int KS>
struct TcShape {
  static constexpr int R = 8 * MB;                 // A rows per patch slot
  static constexpr int N = 16 * G;                 // MMA N
  static constexpr int K = 16 * KS;                // padded K
  static constexpr int DCOLS = N <= 32 ? 32 : 64;  // tensor-memory columns of one accumulator
  static constexpr int TCOLS = 2 * DCOLS;          // two accumulators
  static constexpr int A_KH = 16 * 128;            // K-adjacent core matrices of A (128 rows)
  static constexpr int A_KS = 2 * A_KH;            // one K-step of A
  static constexpr int A_STAGE = KS * A_KS;
  static constexpr int B_KH = (N / 8) * 128;       // K-adjacent core matrices of B
  static constexpr int B_KS = 2 * B_KH;
  static constexpr int B_BYTES = KS * B_KS;
  static constexpr int QN = G * K * 4;             // float4 items (row k of slot j, 4 right-hand sides)
  static constexpr int QI = (QN + 127) / 128;      // items per gather thread
  // shared bytes: A ring, B ring, column maxima, mbarriers, TMEM address and abort flag
  static constexpr int NBAR = 2 * kSA + 2 * kSB + 4;
  static constexpr int SMEM = kSA * A_STAGE + kSB * B_BYTES + kSC * 4 * G * kNR + 8 * NBAR + 16;
  static_assert(G * R <= 128, "patch slots exceed the 128 accumulator lanes");
  static_assert(N % 16 == 0 && N >= 16 && N <= 64, "M = 128 needs N a multiple of 16; two accumulators fit 128 columns");
  static_assert((K * 4) % 32 == 0 && QN % 32 == 0, "a warp's items must share one patch slot");
};

// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort, int* err) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (globaltimer() - t0 > kWaitNs) {
      *abort = 1;
      atomicExch(err, kErrTimeout);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void gather_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// One size class: group g holds the work items lo + G g .. lo + G g + G - 1.
//   gdof[(g G + j) K + k]  DoF of row k of slot j (-1 past the patch or for an empty slot)
//   gpos[g 128 + t]        delta row of accumulator lane t = 8 MB j + r (-1: no patch row)
//   gmeta[g]               (byte offset of the group's A image: low, high word; its bytes; 0)
//   gscale[g G + j]        the patch's inverse scale (its largest |entry|)
// This CTA takes groups blockIdx.x + i gridDim.x, i = 0, 1, ...; group i uses A stage i % kSA,
// B stage i % kSB, column-maximum slot i % kSC and accumulator i % 2.
template <int MB, int G, int KS, bool kHalf>
__global__ void __launch_bounds__(kTcThreadsWs, 3) k_patch_tc(TcClass C, const uint8_t* __restrict__ frag,
                                                               const float* __restrict__ rhs,
                                                               float* __restrict__ delta, int* __restrict__ err,
                                                               int skip_group) {
  using S = TcShape<MB, G, KS>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Abuf = smem;                                                 // [kSA][A_STAGE]
  uint8_t* Bbuf = smem + kSA * S::A_STAGE;                              // [kSB][B_BYTES]
  int* cmax = reinterpret_cast<int*>(Bbuf + kSB * S::B_BYTES);         // [kSC][G][16] float bits >= 0
  uint64_t* bars = reinterpret_cast<uint64_t*>(cmax + kSC * G * kNR);
  uint64_t* afull = bars;                  // [kSA] copies landed (bytes)
  uint64_t* aempty = afull + kSA;          // [kSA] MMAs that read the stage completed
  uint64_t* bfull = aempty + kSA;          // [kSB] 128 gather threads arrived
  uint64_t* bempty = bfull + kSB;          // [kSB] MMAs that read the stage completed
  uint64_t* dfull = bempty + kSB;          // [2] accumulator ready
  uint64_t* dempty = dfull + 2;            // [2] 128 read-back threads done with it
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + S::NBAR);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* gok = reinterpret_cast<volatile int*>(tslot + 2);   // gather warps' shared verdict

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ng = C.ngroups, grid = int(gridDim.x);
  const int n = int(blockIdx.x) < ng ? (ng - 1 - int(blockIdx.x)) / grid + 1 : 0;   // groups of this CTA
  // zero the A ring once: K chunks a patch does not fill keep finite values (zeros or an earlier
  // patch's entries), which the zero rows of its B block cancel
  for (int i = tid; i < kSA * S::A_STAGE / 16; i += kTcThreadsWs) reinterpret_cast<uint4*>(Abuf)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < kSA; ++s) {
      mbar_init(&afull[s], 1);
      mbar_init(&aempty[s], 1);
    }
    for (int s = 0; s < kSB; ++s) {
      mbar_init(&bfull[s], 128);
      mbar_init(&bempty[s], 1);
    }
    for (int d = 0; d < 2; ++d) {
      mbar_init(&dfull[d], 1);
      mbar_init(&dempty[d], 128);
    }
    *abort = 0;
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
  auto gidx = [&](int i) { return int(blockIdx.x) + i * grid; };

  if (warp == 8) {
    // ======================= producer: bulk copies and MMAs (one thread) ========================
    if (lane == 0) {
      int next = 0;                        // next group whose copies are to be issued
      int issued = 0;                      // groups whose MMAs were issued
      bool ok = true;
      for (int i = 0; i < n && ok; ++i) {
        for (; next < n && next < i + kSA; ++next) {
          const int s = next % kSA;
          if (next >= kSA && !mbar_wait_ab(&aempty[s], uint32_t((next / kSA - 1) & 1), abort, err)) {
            ok = false;
            break;
          }
          // the group's A image, K chunk after K chunk (2048 bytes each): one bulk copy.  K chunks
          // beyond it keep an earlier group's finite values, which the zero B rows cancel.
          const int4 m = __ldg(C.gmeta + gidx(next));
          const uint32_t bytes = uint32_t(m.z);
          mbar_expect_tx(&afull[s], bytes);
          // (a test of the bounded waits withholds one announced copy: its barrier never completes)
          if (gidx(next) != skip_group)
            bulk_g2s(Abuf + s * S::A_STAGE, frag + ((int64_t(uint32_t(m.y)) << 32) | uint32_t(m.x)), bytes, &afull[s]);
        }
        if (!ok) break;
        const int sa = i % kSA, sb = i % kSB, d = i & 1;
        if (!mbar_wait_ab(&afull[sa], uint32_t((i / kSA) & 1), abort, err)) break;
        if (!mbar_wait_ab(&bfull[sb], uint32_t((i / kSB) & 1), abort, err)) break;
        if (i >= 2 && !mbar_wait_ab(&dempty[d], uint32_t((i / 2 - 1) & 1), abort, err)) break;
        tc_fence_after();
        const uint32_t a0 = smem_u32(Abuf + sa * S::A_STAGE), b0 = smem_u32(Bbuf + sb * S::B_BYTES);
        constexpr uint32_t idesc = idesc_f16(128, S::N, kHalf);
#pragma unroll
        for (int kk = 0; kk < KS; ++kk)
          tc_mma(tmem + uint32_t(d * S::DCOLS), sdesc(a0 + kk * S::A_KS, S::A_KH, 128),
                 sdesc(b0 + kk * S::B_KS, S::B_KH, 128), idesc, kk > 0 ? 1u : 0u);
        tc_commit(&dfull[d]);
        tc_commit(&aempty[sa]);
        tc_commit(&bempty[sb]);
        issued = i + 1;
      }
      // before the shared and tensor memory are released: the last MMAs and every copy issued
      // (bounded waits; after an abort whatever is still pending gets its chance to land)
      if (issued > 0) {
        const int i = issued - 1;
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&aempty[i % kSA], uint32_t((i / kSA) & 1)) && globaltimer() - t0 < kWaitNs) {
        }
      }
          for (int i = issued; i < next; ++i) {
        if (gidx(i) == skip_group) continue;   // never issued
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&afull[i % kSA], uint32_t((i / kSA) & 1)) && globaltimer() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp >= 4) {
    // ======================= gather: residual rows -> scaled 16-bit B tiles ======================
    const int gt = tid - 128;              // 0..127
    const int gw = gt >> 5;                // gather warp 0..3
    auto load_idx = [&](int i, int (&idx)[S::QI]) {
#pragma unroll
      for (int u = 0; u < S::QI; ++u) {
        const int q = gt + 128 * u;
        idx[u] = (i < n && q < S::QN) ? __ldg(C.gdof + int64_t(gidx(i)) * G * S::K + (q >> 2)) : -1;
      }
    };
    auto load_rhs = [&](const int (&idx)[S::QI], float4 (&v)[S::QI]) {
#pragma unroll
      for (int u = 0; u < S::QI; ++u) {
        const int q = gt + 128 * u;
        v[u] = idx[u] >= 0 ? __ldg(reinterpret_cast<const float4*>(rhs + int64_t(idx[u]) * kNR) + (q & 3))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    float4 cur[S::QI];
    int nidx[S::QI];
    {
      int idx0[S::QI];
      load_idx(0, idx0);
      load_rhs(idx0, cur);
      load_idx(1, nidx);
    }
    for (int i = 0; i < n; ++i) {
      const int sb = i % kSB;
      int* cb = cmax + (i % kSC) * G * kNR;
      uint8_t* Bt = Bbuf + sb * S::B_BYTES;
      // B stage sb and column-maximum slot i % kSC are free once the MMAs of group i - kSB have
      // completed (those were issued after the read-back of group i - 2 kSB released its accumulator).
      // One thread waits and the four warps take its answer together (the named barrier below must
      // see all 128 threads or none).
      if (gt == 0) *gok = (i < kSB || mbar_wait_ab(&bempty[sb], uint32_t((i / kSB - 1) & 1), abort, err)) ? 1 : 0;
      if (kHalf && gt < G * kNR) cb[gt] = 0;
      gather_sync();
      if (!*gok) break;
      // FP16: column maxima (warp maxima over its 8 rows, then shared-memory atomics) to bring each
      // column into FP16's range; BF16 has FP32's exponent range and rounds the columns unscaled
#pragma unroll
      for (int u = 0; u < (kHalf ? S::QI : 0); ++u) {
        const int q0 = 128 * u + gw * 32;  // first item of this warp (warp-uniform)
        if (q0 < S::QN) {
          float m[4] = {fabsf(cur[u].x), fabsf(cur[u].y), fabsf(cur[u].z), fabsf(cur[u].w)};
#pragma unroll
          for (int e = 0; e < 4; ++e)
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) m[e] = fmaxf(m[e], __shfl_xor_sync(0xffffffffu, m[e], o));
          if (lane < 4) {
            const int j = (q0 + lane) / (S::K * 4);
#pragma unroll
            for (int e = 0; e < 4; ++e) atomicMax(cb + j * kNR + 4 * lane + e, __float_as_int(m[e]));
          }
        }
      }
      if (kHalf) gather_sync();
      // scale each column, round to 16 bits: element (n = 16 j + c, k) of the K-major B tile at
      // (k/16) B_KS + ((k/8)%2) B_KH + (n/8) 128 + (n%8) 16 + (k%8) 2
#pragma unroll
      for (int u = 0; u < S::QI; ++u) {
        const int q = gt + 128 * u;
        if (q < S::QN) {
          const int j = q / (S::K * 4), k = (q >> 2) % S::K, c4 = q & 3;
          const float v[4] = {cur[u].x, cur[u].y, cur[u].z, cur[u].w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int nn = 16 * j + 4 * c4 + e;
            float x = v[e];
            if constexpr (kHalf) {
              const float mx = __int_as_float(cb[j * kNR + 4 * c4 + e]);
              x = mx > 0.f ? v[e] * (1.f / mx) : 0.f;
            }
            const int off = (k >> 4) * S::B_KS + ((k >> 3) & 1) * S::B_KH + (nn >> 3) * 128 + (nn & 7) * 16 + (k & 7) * 2;
            if constexpr (kHalf)
              *reinterpret_cast<__half*>(Bt + off) = __float2half_rn(x);
            else
              *reinterpret_cast<__nv_bfloat16*>(Bt + off) = __float2bfloat16_rn(x);
          }
        }
      }
      fence_proxy_async();
      mbar_arrive(&bfull[sb]);
      // the next group's rows (DoF indices loaded one group earlier) and the DoF indices after that
      load_rhs(nidx, cur);
      load_idx(i + 2, nidx);
    }
  } else {
    // ======================= read-back: accumulator lane -> corrections ==========================
    const int t = tid;                     // accumulator lane 0..127
    const int jt = t / S::R < G ? t / S::R : 0;
    for (int i = 0; i < n; ++i) {
      const int d = i & 1, g = gidx(i);
      const int* cb = cmax + (i % kSC) * G * kNR;
      const int prow = __ldg(C.gpos + int64_t(g) * 128 + t);
      const float sa = prow >= 0 ? __ldg(C.gscale + int64_t(g) * G + jt) : 0.f;
      // lane 0 waits, the warp takes its answer (tcgen05.ld below needs all 32 lanes)
      int okw = 0;
      if (lane == 0) okw = mbar_wait_ab(&dfull[d], uint32_t((i / 2) & 1), abort, err) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      tc_fence_after();
      float acc[G][16];
#pragma unroll
      for (int j = 0; j < G; ++j)
        tc_ld16(tmem + (uint32_t(32 * warp) << 16) + uint32_t(d * S::DCOLS + 16 * j), acc[j]);
      tc_wait_ld();
      // the column maxima of this group, read before the accumulator is released: slot i % kSC is
      // rewritten only by the gather of group i + kSC, which waits for MMAs issued after this release
      float cm[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) cm[c] = kHalf ? __int_as_float(cb[jt * kNR + c]) : 1.f;
      tc_fence_before();
      mbar_arrive(&dempty[d]);
      if (prow >= 0) {
        float* o = delta + int64_t(prow) * kNR;
#pragma unroll
        for (int jj = 0; jj < G; ++jj)
          if (jj == jt) {
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
              float4 v;
              v.x = acc[jj][4 * c4 + 0] * (sa * cm[4 * c4 + 0]);
              v.y = acc[jj][4 * c4 + 1] * (sa * cm[4 * c4 + 1]);
              v.z = acc[jj][4 * c4 + 2] * (sa * cm[4 * c4 + 2]);
              v.w = acc[jj][4 * c4 + 3] * (sa * cm[4 * c4 + 3]);
              reinterpret_cast<float4*>(o)[c4] = v;
            }
          }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, S::TCOLS);
}

// Pack the A image of every group: block = one group; 32-bit word w of K chunk c, row block m holds
// columns 8c + 2(w % 4), +1 of row 8m + w / 4 of the 128-row tile; the tile's row r belongs to slot
// j = r / (8 MB) (local row r - 8 MB j).  Values: the FP64 inverse (warp-packed layout of
// kernels_patch.cu) times 1 / ascale[p], zero outside the patch.
template <int MB, int G, bool kHalf>
__global__ void k_pack_tc(TcClass C, const int* __restrict__ slot_ptr, const int64_t* __restrict__ foff64,
                          const double* __restrict__ inv64, const float* __restrict__ ascale,
                          uint8_t* __restrict__ frag) {
  const int g = blockIdx.x;
  const int4 meta = C.gmeta[g];
  const int nchunk = meta.z / 2048;
  uint32_t* dst = reinterpret_cast<uint32_t*>(frag + ((int64_t(uint32_t(meta.y)) << 32) | uint32_t(meta.x)));
  for (int e = threadIdx.x; e < nchunk * 16 * 32; e += blockDim.x) {
    const int c = e >> 9, m = (e >> 5) & 15, w = e & 31;
    const int row = 8 * m + (w >> 2), col = 8 * c + 2 * (w & 3);
    const int j = row / (8 * MB), lr = row - 8 * MB * j;
    double v0 = 0.0, v1 = 0.0;
    if (j < G) {
      const int2 sl = C.gslot[int64_t(g) * G + j];
      const int n = sl.x, p = sl.y;
      if (n > 0 && lr < n) {
        const int NB4 = (n + 3) / 4;
        const double* src = inv64 + foff64[p];
        const double inv = 1.0 / double(ascale[p]);
        auto at = [&](int cc) -> double {
          return cc < n ? src[((lr >> 3) * NB4 + (cc >> 2)) * 32 + (lr & 7) + 8 * (cc & 3)] * inv : 0.0;
        };
        v0 = at(col);
        v1 = at(col + 1);
      }
    }
    dst[e] = pack2<kHalf>(float(v0), float(v1));
  }
}

__global__ void k_tc_fill_scale(int nslot, const int2* __restrict__ gslot, const float* __restrict__ ascale,
                                float* __restrict__ gscale) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nslot) return;
  const int2 m = gslot[e];
  gscale[e] = m.x > 0 ? ascale[m.y] : 0.f;
}

template <int MB, int G, int KS, bool kHalf>
int launch_tc(const TcPatches& T, int c, const float* rhs, float* delta, int* err, int skip_group, cudaStream_t s) {
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
  int occ = 65536 / (regs * kTcThreadsWs);
  occ = std::min(occ, (228 * 1024) / (S::SMEM + int(fa.sharedSizeBytes) + 1024));
  occ = std::min(occ, 2048 / kTcThreadsWs);
  occ = std::min(occ, 512 / S::TCOLS);
  occ = std::max(occ, 1);
  const int grid = C.ngroups < occ * T.nsm ? C.ngroups : occ * T.nsm;
  kern<<<grid, kTcThreadsWs, S::SMEM, s>>>(C, T.frag, rhs, delta, err, skip_group);
  return 1;
}

}  // namespace

int pack_tc(const Patches& P, const TcPatches& T, const double* inv64, const float* ascale, bool half, cudaStream_t s) {
  int k = 0;
  uint8_t* frag = const_cast<uint8_t*>(T.frag);
  for (int c = 0; c < 3; ++c) {
    const TcClass& C = T.cls[c];
    if (C.ngroups <= 0) continue;
#define VK_PACK(MB, G)                                                                                              \
  do {                                                                                                            \
    if (half)                                                                                                     \
      k_pack_tc<MB, G, true><<<C.ngroups, 256, 0, s>>>(C, P.slot_ptr, P.foff, inv64, ascale, frag);               \
    else                                                                                                          \
      k_pack_tc<MB, G, false><<<C.ngroups, 256, 0, s>>>(C, P.slot_ptr, P.foff, inv64, ascale, frag);              \
  } while (0)
    if (c == 0) VK_PACK(5, 3);
    else if (c == 1) VK_PACK(8, 2);
    else VK_PACK(16, 1);
#undef VK_PACK
    const int nslot = C.ngroups * kTcG[c];
    k_tc_fill_scale<<<(nslot + 255) / 256, 256, 0, s>>>(nslot, C.gslot, ascale, const_cast<float*>(C.gscale));
    k += 2;
  }
  return k;
}

int patch_apply_tc(const TcPatches& T, bool half, const float* rhs, float* delta, int* err, int skip_group,
                   cudaStream_t s) {
  // the withheld copy (a test of the bounded waits) belongs to the first launch only
  int k = 0;
  if (half) {
    k += launch_tc<16, 1, 8, true>(T, 2, rhs, delta, err, k == 0 ? skip_group : -1, s);
    k += launch_tc<8, 2, 4, true>(T, 1, rhs, delta, err, k == 0 ? skip_group : -1, s);
    k += launch_tc<5, 3, 3, true>(T, 0, rhs, delta, err, k == 0 ? skip_group : -1, s);
  } else {
    k += launch_tc<16, 1, 8, false>(T, 2, rhs, delta, err, k == 0 ? skip_group : -1, s);
    k += launch_tc<8, 2, 4, false>(T, 1, rhs, delta, err, k == 0 ? skip_group : -1, s);
    k += launch_tc<5, 3, 3, false>(T, 0, rhs, delta, err, k == 0 ? skip_group : -1, s);
  }
  return k;
}

}  // namespace gpu
}  // namespace vk
