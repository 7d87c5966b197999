// C ABI of the Vanka multigrid library (include/vk.h): hierarchy setup, the V-cycle, FGMRES and the
// export calls.  Host orchestration only; every numerical step on the device is a kernel of
// kernels_*.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "gpu.h"
#include "vk.h"
#include "vk_internal.h"

namespace {

thread_local std::string g_err;

// Library-wide lock around the operations that allocate, free or synchronise the whole device, and
// around stream capture: a device-wide synchronisation or a free issued by one thread while another
// thread captures a graph would invalidate that capture.  Solves (launches, copies and waits on the
// caller's stream) never take it, so concurrent solves on different hierarchies still overlap.
std::mutex g_device_mu;

struct VkError {
  int code;
  std::string msg;
};

[[noreturn]] void raise(int code, const std::string& msg) { throw VkError{code, msg}; }

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) raise(VK_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call) ck((call), #call)

template <class F>
int guard(F&& f) {
  try {
    g_err.clear();
    return f();
  } catch (const VkError& e) {
    g_err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return VK_ERR_NO_MEMORY;
  } catch (const std::exception& e) {
    g_err = e.what();
    return VK_ERR_INTERNAL;
  }
}

inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// Device memory through the caller's allocator (or cudaMalloc).  Counts bytes so vk_footprint can be
// checked against what setup really allocates.
struct DeviceMemory {
  vk_allocator user{};
  bool custom = false;
  cudaStream_t stream = nullptr;
  std::vector<void*> live;
  size_t total = 0;
  bool counting_only = false;

  void* get(size_t bytes) {
    bytes = round256(std::max<size_t>(bytes, 1));
    total += bytes;
    if (counting_only) return nullptr;
    void* p = nullptr;
    if (custom) {
      p = user.alloc(user.ctx, bytes, stream);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (!p) raise(VK_ERR_NO_MEMORY, "device allocation of " + std::to_string(bytes) + " bytes failed");
    live.push_back(p);
    return p;
  }
  template <class T>
  T* get_n(size_t n) {
    return static_cast<T*>(get(n * sizeof(T)));
  }
  template <class T>
  T* upload(const std::vector<T>& v) {
    T* p = get_n<T>(v.size());
    if (!counting_only && !v.empty())
      CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, stream));
    return p;
  }
  void release_all() {
    for (void* p : live) {
      if (custom)
        user.release(user.ctx, p, stream);
      else
        cudaFree(p);
    }
    live.clear();
  }
};

struct HostSell {
  std::vector<int64_t> sptr;
  std::vector<int> sw, col, rowof;
  std::vector<double> val;
};

// Threads per row for a SELL matrix: the smallest of 1, 2, 4, 8 that gives at least `warps_per_sm`
// warps per SM (GB300: 152 SMs), so load latency is hidden without an over-long per-thread
// dependency chain.
int sell_tpr(int nrows, int warps_per_sm) {
  const int64_t want = 152LL * warps_per_sm * 32;
  for (int t = 1; t < 8; t *= 2)
    if (int64_t(nrows) * t >= want) return t;
  return 8;
}

// SELL-C: permute rows by decreasing length inside windows of 1024 rows, cut into slices of C rows.
HostSell build_sell(const vk::HostCsr& A, int tpr) {
  HostSell S;
  const int n = A.nrows, W = 1024, C = 32 / tpr;
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  for (int w0 = 0; w0 < n; w0 += W) {
    const int w1 = std::min(n, w0 + W);
    std::stable_sort(order.begin() + w0, order.begin() + w1, [&](int a, int b) {
      return (A.ptr[a + 1] - A.ptr[a]) > (A.ptr[b + 1] - A.ptr[b]);
    });
  }
  const int ns = (n + C - 1) / C;
  S.rowof.assign(size_t(ns) * C, -1);
  for (int i = 0; i < n; ++i) S.rowof[i] = order[i];
  S.sptr.assign(ns + 1, 0);
  S.sw.assign(ns, 0);
  for (int s = 0; s < ns; ++s) {
    int w = 0;
    for (int t = 0; t < C; ++t) {
      const int row = S.rowof[size_t(s) * C + t];
      if (row >= 0) w = std::max(w, A.ptr[row + 1] - A.ptr[row]);
    }
    w = (w + tpr - 1) / tpr * tpr;
    S.sw[s] = w;
    S.sptr[s + 1] = S.sptr[s] + int64_t(C) * w;
  }
  S.col.assign(S.sptr[ns], 0);
  S.val.assign(S.sptr[ns], 0.0);
  for (int s = 0; s < ns; ++s)
    for (int t = 0; t < C; ++t) {
      const int row = S.rowof[size_t(s) * C + t];
      const int len = row >= 0 ? A.ptr[row + 1] - A.ptr[row] : 0;
      for (int k = 0; k < S.sw[s]; ++k) {
        const int64_t pos = S.sptr[s] + int64_t(C) * k + t;
        if (k < len) {
          S.col[pos] = A.col[A.ptr[row] + k];
          S.val[pos] = A.val[A.ptr[row] + k];
        } else {
          // padding: value 0 at a valid column of x (the row itself when the matrix is square,
          // else column 0: P has more rows than the coarse vector has entries)
          S.col[pos] = (row >= 0 && row < A.ncols) ? row : 0;
          S.val[pos] = 0.0;
        }
      }
    }
  for (const int c : S.col)
    if (c < 0 || c >= A.ncols) raise(VK_ERR_INTERNAL, "SELL column out of range");
  return S;
}

struct HostPatchPlan {
  std::vector<int> work;        // canonical ids in processing order
  std::vector<int64_t> foff;    // canonical id -> packed offset
  int64_t ftotal = 0;
  int nb_max = 0;
  bool sym = false;             // symmetric tile layout of the inverses
  int cls_lo[vk::gpu::kApplyClasses] = {}, cls_hi[vk::gpu::kApplyClasses] = {};  // work-list range of each size class
  std::vector<int> dof_ptr, slot_pos;
  std::vector<double> weight;
};

// Work order, storage offsets and DoF -> slot transpose of one level's patches.  FP32 and FP32-pair
// inverses use the symmetric tile layout when every patch of the level has at most kSymMaxN DoFs.
HostPatchPlan plan_patches(const vk::HostLevel& L, int weights, int prec) {
  HostPatchPlan P;
  const int np = int(L.patch_ptr.size()) - 1;
  P.work.resize(np);
  std::iota(P.work.begin(), P.work.end(), 0);
  auto nb = [&](int p) { return (L.patch_ptr[p + 1] - L.patch_ptr[p] + 3) / 4; };
  std::stable_sort(P.work.begin(), P.work.end(), [&](int a, int b) { return nb(a) > nb(b); });
  int nmax = 0;
  for (int p = 0; p < np; ++p) nmax = std::max(nmax, L.patch_ptr[p + 1] - L.patch_ptr[p]);
  P.sym = prec != VK_PREC_F64 && nmax <= vk::gpu::kSymMaxN;
  P.foff.assign(np, 0);
  for (int w = 0; w < np; ++w) {
    const int p = P.work[w];
    const int n = L.patch_ptr[p + 1] - L.patch_ptr[p];
    P.foff[p] = P.ftotal;
    P.ftotal += P.sym ? vk::gpu::sym_packed_size(n) : vk::gpu::packed_size(n);
    P.nb_max = std::max(P.nb_max, nb(p));
  }
  // size classes of ceil(n/4) (the work list is sorted by it, largest first, so each class is a range)
  for (int c = 0; c < vk::gpu::kApplyClasses; ++c) {
    const int lo = c == 0 ? 1 : vk::gpu::kApplyClassHi[c - 1] + 1, hi = vk::gpu::kApplyClassHi[c];
    int a = np, b = 0;
    for (int w = 0; w < np; ++w) {
      const int v = nb(P.work[w]);
      if (v >= lo && v <= hi) {
        a = std::min(a, w);
        b = std::max(b, w + 1);
      }
    }
    P.cls_lo[c] = a < b ? a : 0;
    P.cls_hi[c] = a < b ? b : 0;
  }
  if (P.nb_max > vk::gpu::kApplyClassHi[vk::gpu::kApplyClasses - 1])
    raise(VK_ERR_ARG, "patches larger than 168 DoFs are not supported");
  const int64_t nslots = L.patch_dofs.size();
  P.dof_ptr.assign(L.ndof + 1, 0);
  for (int64_t s = 0; s < nslots; ++s) P.dof_ptr[L.patch_dofs[s] + 1]++;
  for (int i = 0; i < L.ndof; ++i) P.dof_ptr[i + 1] += P.dof_ptr[i];
  P.slot_pos.assign(nslots, 0);
  std::vector<int> fill(P.dof_ptr.begin(), P.dof_ptr.end() - 1);
  for (int64_t s = 0; s < nslots; ++s) P.slot_pos[s] = fill[L.patch_dofs[s]]++;
  if (weights == VK_WEIGHTS_MULTIPLICITY) {
    P.weight.assign(L.ndof, 1.0);
    for (int i = 0; i < L.ndof; ++i) {
      const int c = P.dof_ptr[i + 1] - P.dof_ptr[i];
      if (c > 0) P.weight[i] = 1.0 / c;
    }
  }
  return P;
}

struct DevLevel {
  int N = 0, ndof = 0, n_u = 0, n_p = 0;
  vk::gpu::Sell A, P, R;   // level matrix; prolongation from / restriction to the coarser level
  vk::gpu::Csr Acsr;
  uint8_t* dir = nullptr;
  vk::gpu::Patches pat;
  double lam = 0.0;
  double *b = nullptr, *x = nullptr, *r = nullptr, *d = nullptr, *t = nullptr, *delta = nullptr;
  float2* r2 = nullptr;  // FP32-pair residual (emulated-FP64 inverses only)
  vk::gpu::PatchElems pe;   // element data of the matrix-free patch assembly (patch_assembly = 1)
  // multi-right-hand-side structures (batch_prec != VK_BATCH_NONE)
  vk::gpu::SellB Ab, Pb, Rb;                 // SELL-8 copies for the 16-right-hand-side products
  int64_t* foff16 = nullptr;
  void* frag = nullptr;
  float* ascale = nullptr;
  int mt_max = 0;
  vk::gpu::TcPatches tc;                     // tcgen05 path: core-matrix inverses and size classes
  double tc_bytes = 0.0;                     // bytes of all A images of the level
  float *bb = nullptr, *xb = nullptr, *rb = nullptr, *db = nullptr, *delta_f = nullptr;
};

// Outcome of the patch-apply autotuner on one level: the chosen candidate and every candidate's
// best time (microseconds; 0 when not timed).
struct TuneResult {
  int index = 3;        // default shape: one launch, 256 threads, one warp per patch
  double us[16] = {};
};

// Pairs of CUDA events recorded on the launching stream around selected kernels; the summed
// durations are read by vk_stats_read.
struct KTimer {
  std::vector<cudaEvent_t> ev;
  size_t used = 0;
  void begin(cudaStream_t s) {
    if (used + 2 > ev.size())
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        ev.push_back(e);
      }
    CK(cudaEventRecord(ev[used], s));
  }
  void end(cudaStream_t s) {
    CK(cudaEventRecord(ev[used + 1], s));
    used += 2;
  }
  int64_t count() const { return int64_t(used / 2); }
  double total_ms() const {
    double ms = 0.0;
    for (size_t i = 0; i + 1 < used; i += 2) {
      CK(cudaEventSynchronize(ev[i + 1]));
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
      ms += t;
    }
    return ms;
  }
  ~KTimer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

}  // namespace

struct vk_hierarchy {
  vk_problem prob{};
  vk_options opt{};
  std::vector<vk::HostLevel> host;
  std::vector<DevLevel> lv;
  DeviceMemory mem;
  bool host_only = false;
  int nc = 0;
  double* Cinv = nullptr;
  int kmax = 0;
  int64_t ldv = 0;
  double *V = nullptr, *Z = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *hist = nullptr;
  double *yv = nullptr, *t2 = nullptr, *partial = nullptr, *scal = nullptr;
  double *bh = nullptr, *xh = nullptr;
  int* iflag = nullptr;
  int* h_flag = nullptr;     // pinned host mirror (2 ints)
  double* h_scal = nullptr;  // pinned host mirror (4 doubles)
  std::vector<double> lambdas;
  // statistics (vk_stats_*)
  int64_t n_launch = 0, n_vcycle = 0;
  bool time_apply = false;
  std::vector<TuneResult> tune;  // per level (index 0 unused)
  KTimer tm_apply;   // finest-level patch applications
  KTimer tm_spmv;    // finest-level V-cycle residual SpMV (SELL, or the block SpMM of vk_solve_batch)
  double apply_bytes = 0.0, apply_flops = 0.0;
  double bapply_bytes = 0.0, bapply_flops = 0.0;
  double spmv_bytes = 0.0, bspmv_bytes = 0.0;
  double factor_ms = 0.0, setup_ms = 0.0;
  // graph-resident FGMRES (one CUDA graph per hierarchy: prologue, WHILE node, epilogue)
  vk::gpu::FgState* st = nullptr;        // device
  vk::gpu::FgState* h_par = nullptr;     // pinned: parameters written before each launch
  vk::gpu::FgState* h_res = nullptr;     // pinned: state copied back by the graph
  double* h_hist = nullptr;              // pinned: residual history copied back by the graph
  double *vin = nullptr, *zbuf = nullptr, *wbuf = nullptr;
  cudaStream_t cap0 = nullptr, cap1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  int64_t g_pro = 0, g_body = 0, g_epi = 0;   // kernels per prologue / iteration / epilogue
  int graph_pdl = 0;                          // 1: the graph was captured with programmatic launches
  // vk_solve_batch workspace (finest level, FP64, 16 interleaved right-hand sides)
  int kb = 0;
  int64_t ldb = 0;
  float* cinv_f = nullptr;                    // FP32 coarse inverse (batch_coarse_fp32)
  double *cb64 = nullptr, *cx64 = nullptr;     // FP64 coarse right-hand sides / solutions (batch)
  double *Vb = nullptr, *Zb = nullptr, *wb = nullptr, *xob = nullptr, *Hb = nullptr, *csb = nullptr, *snb = nullptr;
  double *gb = nullptr, *histb = nullptr, *hcolb = nullptr, *t2b = nullptr, *partb = nullptr, *sqb = nullptr;
  double* yb = nullptr;
  int *activeb = nullptr, *itersb = nullptr, *nonfb = nullptr;
  int* tc_err = nullptr;   // set by the tcgen05 patch solves when a bounded wait expires
  bool in_group = false;   // the FGMRES workspace is used by a vk_group member
  bool expire_once = false;  // vk_options.test_expire_wait, consumed by the first finest sweep
  ~vk_hierarchy() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (cap0) cudaStreamDestroy(cap0);
    if (cap1) cudaStreamDestroy(cap1);
    if (h_par) cudaFreeHost(h_par);
    if (h_res) cudaFreeHost(h_res);
    if (h_hist) cudaFreeHost(h_hist);
  }
};

namespace {

// Candidate launch shapes of the patch application (see vk::gpu::ApplySched).
std::vector<vk::gpu::ApplySched> apply_candidates() {
  std::vector<vk::gpu::ApplySched> c;
  for (int split = 0; split < 2; ++split)
    for (int threads : {128, 256})
      for (int per_sm : {0, 4, 8}) c.push_back({split, threads, per_sm});
  return c;
}

void validate(const vk_problem* p, const vk_options* o) {
  if (!p || !o) raise(VK_ERR_ARG, "null problem or options");
  if (p->cell != VK_CELL_TRIANGLE && p->cell != VK_CELL_QUAD && p->cell != VK_CELL_BDM)
    raise(VK_ERR_ARG, "cell must be VK_CELL_TRIANGLE, VK_CELL_QUAD or VK_CELL_BDM");
  if (p->cell == VK_CELL_BDM) {
    if (p->k < 1 || p->k > 5) raise(VK_ERR_ARG, "BDM order k must be in 1..5");
  } else if (p->k < 2 || p->k > 4) {
    raise(VK_ERR_ARG, "order k must be 2, 3 or 4");
  }
  if (p->N_coarse < 1 || p->nlevels < 1 || p->nlevels > 12) raise(VK_ERR_ARG, "bad mesh hierarchy");
  const int64_t Nf = int64_t(p->N_coarse) << (p->nlevels - 1);
  if (Nf * p->k > 8192) raise(VK_ERR_ARG, "finest mesh too large for 32-bit indices");
  if (p->cell == VK_CELL_BDM) {
    // (k+1)(k+2) velocity functions per cell; an edge row couples at most the six cells around the two
    // cells of its edge, plus their pressures
    const int64_t nb = int64_t(p->k + 1) * (p->k + 2), nq = int64_t(p->k) * (p->k + 1) / 2;
    const int64_t ncell = 2 * Nf * Nf, n_u = 3 * Nf * Nf * (p->k + 1) + ncell * (p->k + 1) * (p->k - 1);
    if (n_u * (6 * nb + 2 * nq) + ncell * nq * nb > int64_t(INT32_MAX))
      raise(VK_ERR_ARG, "finest BDM mesh too large for 32-bit indices");
  }
  if (!(p->nu > 0.0) || !std::isfinite(p->nu)) raise(VK_ERR_ARG, "viscosity must be positive and finite");
  if (p->bc != VK_BC_DIRICHLET_ALL) raise(VK_ERR_ARG, "bc must be VK_BC_DIRICHLET_ALL");
  {
    const double* d = p->domain;
    const bool unset = d[0] == 0.0 && d[1] == 0.0 && d[2] == 0.0 && d[3] == 0.0;
    const bool unit = d[0] == 0.0 && d[1] == 1.0 && d[2] == 0.0 && d[3] == 1.0;
    if (!unset && !unit) raise(VK_ERR_ARG, "domain must be the unit square {0, 1, 0, 1}");
  }
  if (o->sweeps < 1) raise(VK_ERR_ARG, "sweeps must be >= 1");
  if (o->weights != VK_WEIGHTS_PLAIN && o->weights != VK_WEIGHTS_MULTIPLICITY) raise(VK_ERR_ARG, "bad weights");
  if (o->factor_prec != VK_PREC_F64 && o->factor_prec != VK_PREC_F32 && o->factor_prec != VK_PREC_F64E)
    raise(VK_ERR_ARG, "bad factor_prec");
  if (!(o->cheb_hi > o->cheb_lo) || !(o->cheb_lo > 0.0)) raise(VK_ERR_ARG, "bad Chebyshev interval");
  if (o->eig_steps < 1 || o->eig_steps > 64) raise(VK_ERR_ARG, "eig_steps must be in 1..64");
  if (o->max_iterations < 1 || o->max_iterations > 1000) raise(VK_ERR_ARG, "max_iterations must be in 1..1000");
  if (o->batch_prec < VK_BATCH_NONE || o->batch_prec > VK_BATCH_FP16) raise(VK_ERR_ARG, "bad batch_prec");
  if (o->batch_engine != VK_ENGINE_TCGEN05 && o->batch_engine != VK_ENGINE_MMA_SYNC) raise(VK_ERR_ARG, "bad batch_engine");
  if (o->test_expire_wait != 0 && o->test_expire_wait != 1) raise(VK_ERR_ARG, "test_expire_wait must be 0 or 1");
  if (o->spmv_warps < 1 || o->spmv_warps > 4096) raise(VK_ERR_ARG, "spmv_warps must be in 1..4096");
  if (o->batch_coarse_fp32 != 0 && o->batch_coarse_fp32 != 1) raise(VK_ERR_ARG, "batch_coarse_fp32 must be 0 or 1");
  if (o->test_singular_patch < -1) raise(VK_ERR_ARG, "test_singular_patch must be -1 or a patch id");
  if (o->graph_pdl != 0 && o->graph_pdl != 1) raise(VK_ERR_ARG, "graph_pdl must be 0 or 1");
  if (o->patch_assembly != VK_ASSEMBLY_MATRIX_FULL && o->patch_assembly != VK_ASSEMBLY_MATRIX_FREE)
    raise(VK_ERR_ARG, "bad patch_assembly");
  if (p->cell == VK_CELL_BDM && o->patch_assembly != VK_ASSEMBLY_MATRIX_FULL)
    raise(VK_ERR_ARG, "BDM patches are gathered from the assembled matrix (VK_ASSEMBLY_MATRIX_FULL)");
  if (o->apply_schedule < -1 || o->apply_schedule >= int(apply_candidates().size()))
    raise(VK_ERR_ARG, "apply_schedule must be -1 or a candidate index");
  if (o->batch_prec != VK_BATCH_NONE) {
    if (o->factor_prec != VK_PREC_F64) raise(VK_ERR_ARG, "batch_prec needs FP64 factor_prec");
    if (o->batch_max_iterations < 1 || o->batch_max_iterations > 127)
      raise(VK_ERR_ARG, "batch_max_iterations must be in 1..127");
  }
}

void build_host(vk_hierarchy* h) {
  const int L = h->prob.nlevels;
  int nthreads = h->opt.host_threads > 0 ? h->opt.host_threads : int(std::thread::hardware_concurrency());
  nthreads = std::max(1, std::min(nthreads, 64));
  h->host.resize(L);
  for (int l = 0; l < L; ++l) {
    vk::build_level(h->prob.N_coarse << l, h->prob.k, h->prob.nu, l > 0, nthreads, h->host[l],
                    l > 0 && h->opt.patch_assembly == VK_ASSEMBLY_MATRIX_FREE, h->prob.cell);
    if (l > 0) vk::build_transfer(h->host[l - 1], h->host[l]);
  }
}

vk::gpu::Sell upload_sell(DeviceMemory& m, const vk::HostCsr& A, int warps_per_sm) {
  const int tpr = sell_tpr(A.nrows, warps_per_sm);
  HostSell S = build_sell(A, tpr);
  vk::gpu::Sell d;
  d.tpr = tpr;
  d.nrows = A.nrows;
  d.nslices = int(S.sw.size());
  d.sptr = m.upload(S.sptr);
  d.swidth = m.upload(S.sw);
  d.col = m.upload(S.col);
  d.val = m.upload(S.val);
  d.rowof = m.upload(S.rowof);
  return d;
}

// CSR copy on the device.  zero_row >= 0 uploads that row with zero values (test of the
// singular-patch path only; the host matrix is unchanged).
vk::gpu::Csr upload_csr(DeviceMemory& m, const vk::HostCsr& A, int zero_row = -1) {
  vk::gpu::Csr c;
  c.nrows = A.nrows;
  c.ptr = m.upload(A.ptr);
  c.col = m.upload(A.col);
  if (zero_row >= 0 && zero_row < A.nrows) {
    std::vector<double> v(A.val);
    for (int e = A.ptr[zero_row]; e < A.ptr[zero_row + 1]; ++e) v[e] = 0.0;
    c.val = m.upload(v);
  } else {
    c.val = m.upload(A.val);
  }
  return c;
}

// SELL-8 copy of a matrix for the 16-right-hand-side products: FP32 values, and FP64 values too when
// `fp64` (the finest matrix, used by the FP64 outer iteration).
vk::gpu::SellB upload_sell8(DeviceMemory& m, const vk::HostCsr& A, bool fp64) {
  const HostSell S = build_sell(A, 4);   // 4 threads per row in the SELL builder = slices of 8 rows
  vk::gpu::SellB d;
  d.nrows = A.nrows;
  d.nslices = int(S.sw.size());
  d.sptr = m.upload(S.sptr);
  d.swidth = m.upload(S.sw);
  d.col = m.upload(S.col);
  d.rowof = m.upload(S.rowof);
  std::vector<float> vf(S.val.size());
  for (size_t i = 0; i < vf.size(); ++i) vf[i] = float(S.val[i]);
  d.valf = m.upload(vf);
  if (fp64) d.vald = m.upload(S.val);
  return d;
}

// Multi-right-hand-side structures: FP32 copies of the matrices, CSR transfers, 16-bit patch
// fragments, FP32 block vectors per level, the FP32 coarse inverse and the FP64 batched Krylov bases.
void allocate_batch(vk_hierarchy* h) {
  DeviceMemory& m = h->mem;
  const int L = h->prob.nlevels;
  constexpr int NR = 16;
  for (int l = 0; l < L; ++l) {
    const vk::HostLevel& H = h->host[l];
    DevLevel& D = h->lv[l];
    D.Ab = upload_sell8(m, H.A, l == L - 1);
    if (l > 0) {
      D.Pb = upload_sell8(m, H.P, false);
      D.Rb = upload_sell8(m, H.R, false);
      const int np = int(H.patch_ptr.size()) - 1;
      std::vector<int64_t> f16(np);
      int64_t tot = 0;
      int mt = 0;
      for (int p = 0; p < np; ++p) {
        const int n = H.patch_ptr[p + 1] - H.patch_ptr[p];
        f16[p] = tot;
        tot += vk::gpu::frag_size(n);
        mt = std::max(mt, (n + 15) / 16);
      }
      if (mt > 8) raise(VK_ERR_ARG, "patches larger than 128 are not supported by the batched path");
      D.mt_max = mt;
      D.foff16 = m.upload(f16);
      D.frag = m.get(size_t(tot) * 16);
      D.ascale = m.get_n<float>(np);
      // tcgen05 layout: size classes n <= 40, 64, 128 are ranges of the work list (sorted by ceil(n/4),
      // largest first), cut into groups of kTcG[c] patches; each group's A image holds ceil(nmax/8)
      // K chunks of 2048 bytes
      {
        const HostPatchPlan plan = plan_patches(H, h->opt.weights, h->opt.factor_prec);
        int64_t btot = 0;
        vk::gpu::TcPatches& T = D.tc;
        for (int c = 0; c < 3; ++c) {
          int lo = np, hi = 0;
          for (int w = 0; w < np; ++w) {
            const int pw = plan.work[w], n = H.patch_ptr[pw + 1] - H.patch_ptr[pw];
            if (n <= vk::gpu::kTcCap[c] && (c == 0 || n > vk::gpu::kTcCap[c - 1])) {
              lo = std::min(lo, w);
              hi = std::max(hi, w + 1);
            }
          }
          if (lo >= hi) continue;
          const int G = vk::gpu::kTcG[c], K = vk::gpu::kTcK[c], R = 128 / G / 8 * 8;
          const int ng = (hi - lo + G - 1) / G;
          std::vector<int> gdof(size_t(ng) * G * K, -1), gpos(size_t(ng) * 128, -1);
          std::vector<int2> gslot(size_t(ng) * G, make_int2(0, 0));
          std::vector<int4> gmeta(size_t(ng), make_int4(0, 0, 0, 0));
          for (int g = 0; g < ng; ++g) {
            int nmax = 0;
            for (int j = 0; j < G; ++j) {
              const int w = lo + g * G + j;
              if (w >= hi) break;
              const int pw = plan.work[w], s0 = H.patch_ptr[pw], n = H.patch_ptr[pw + 1] - s0;
              for (int k = 0; k < n; ++k) {
                gdof[(size_t(g) * G + j) * K + k] = H.patch_dofs[s0 + k];
                gpos[size_t(g) * 128 + R * j + k] = plan.slot_pos[s0 + k];
              }
              gslot[size_t(g) * G + j] = make_int2(n, pw);
              nmax = std::max(nmax, n);
            }
            const int64_t bytes = vk::gpu::tc_group_bytes(nmax);
            gmeta[g] = make_int4(int(uint32_t(uint64_t(btot))), int(uint32_t(uint64_t(btot) >> 32)), int(bytes), 0);
            btot += bytes;
          }
          T.cls[c].ngroups = ng;
          T.cls[c].gdof = m.upload(gdof);
          T.cls[c].gpos = m.upload(gpos);
          T.cls[c].gslot = m.upload(gslot);
          T.cls[c].gmeta = m.upload(gmeta);
          T.cls[c].gscale = m.get_n<float>(size_t(ng) * G);
        }
        T.frag = static_cast<const uint8_t*>(m.get(size_t(btot)));
        D.tc_bytes = double(btot);
      }
      D.delta_f = m.get_n<float>(size_t(H.patch_dofs.size()) * NR);
    }
    D.bb = m.get_n<float>(size_t(H.ndof) * NR);
    D.xb = m.get_n<float>(size_t(H.ndof) * NR);
    D.rb = m.get_n<float>(size_t(H.ndof) * NR);
    D.db = m.get_n<float>(size_t(H.ndof) * NR);
  }
  const int mdim = h->nc + 1;
  if (h->opt.batch_coarse_fp32) {
    h->cinv_f = m.get_n<float>(size_t(mdim) * mdim);
  } else {
    h->cb64 = m.get_n<double>(size_t(h->nc) * NR);
    h->cx64 = m.get_n<double>(size_t(h->nc) * NR);
  }
  const int nf = h->host[L - 1].ndof;
  h->kb = h->opt.batch_max_iterations;
  const int ldh = h->kb + 1;
  h->ldb = int64_t(nf) * NR;
  h->Vb = m.get_n<double>(size_t(h->ldb) * (h->kb + 1));
  h->Zb = m.get_n<double>(size_t(h->ldb) * h->kb);
  h->wb = m.get_n<double>(size_t(h->ldb));
  h->xob = m.get_n<double>(size_t(h->ldb));
  h->Hb = m.get_n<double>(size_t(NR) * ldh * h->kb);
  h->csb = m.get_n<double>(size_t(NR) * ldh);
  h->snb = m.get_n<double>(size_t(NR) * ldh);
  h->gb = m.get_n<double>(size_t(NR) * ldh);
  h->histb = m.get_n<double>(size_t(NR) * ldh);
  h->hcolb = m.get_n<double>(size_t(NR) * ldh);
  h->t2b = m.get_n<double>(size_t(NR) * ldh);
  h->partb = m.get_n<double>(size_t(NR) * ldh * vk::gpu::kBatchBlocks);
  h->sqb = m.get_n<double>(4 * NR);
  h->yb = m.get_n<double>(size_t(NR) * ldh);
  h->activeb = m.get_n<int>(NR);
  h->tc_err = m.get_n<int>(4);
  h->itersb = m.get_n<int>(NR);
  h->nonfb = m.get_n<int>(NR);
}

// Allocates every device buffer (or only counts the bytes when mem.counting_only is set).
void allocate_device(vk_hierarchy* h) {
  DeviceMemory& m = h->mem;
  const int L = h->prob.nlevels;
  h->lv.assign(L, DevLevel{});
  const int fsz = h->opt.factor_prec == VK_PREC_F32 ? 4 : 8;   // FP64 and FP32 pairs: 8 bytes
  for (int l = 0; l < L; ++l) {
    const vk::HostLevel& H = h->host[l];
    DevLevel& D = h->lv[l];
    D.N = H.N;
    D.ndof = H.ndof;
    D.n_u = H.n_u;
    D.n_p = H.n_p;
    D.A = upload_sell(m, H.A, h->opt.spmv_warps);
    int zero_row = -1;
    if (l == L - 1 && h->opt.test_singular_patch >= 0) {
      const int np = int(H.patch_ptr.size()) - 1;
      if (h->opt.test_singular_patch >= np) raise(VK_ERR_ARG, "test_singular_patch out of range");
      zero_row = H.patch_dofs[H.patch_ptr[h->opt.test_singular_patch + 1] - 1];
    }
    D.Acsr = upload_csr(m, H.A, zero_row);
    D.dir = m.upload(H.dir);
    if (l > 0) {
      D.P = upload_sell(m, H.P, h->opt.spmv_warps);
      D.R = upload_sell(m, H.R, h->opt.spmv_warps);
    }
    D.b = m.get_n<double>(H.ndof);
    D.x = m.get_n<double>(H.ndof);
    D.r = m.get_n<double>(H.ndof);
    D.d = m.get_n<double>(H.ndof);
    D.t = m.get_n<double>(H.ndof);
    if (l > 0) {
      HostPatchPlan P = plan_patches(H, h->opt.weights, h->opt.factor_prec);
      vk::gpu::Patches& G = D.pat;
      G.npatch = int(H.patch_ptr.size()) - 1;
      G.ndof = H.ndof;
      G.nslots = int64_t(H.patch_dofs.size());
      G.slot_ptr = m.upload(H.patch_ptr);
      G.slot_dofs = m.upload(H.patch_dofs);
      G.work = m.upload(P.work);
      G.foff = m.upload(P.foff);
      G.factors = m.get(size_t(P.ftotal) * fsz);
      G.prec = h->opt.factor_prec;
      G.nb_max = P.nb_max;
      G.sym = P.sym ? 1 : 0;
      for (int c = 0; c < vk::gpu::kApplyClasses; ++c) {
        G.cls_lo[c] = P.cls_lo[c];
        G.cls_hi[c] = P.cls_hi[c];
      }
      G.dof_ptr = m.upload(P.dof_ptr);
      G.slot_pos = m.upload(P.slot_pos);
      G.weight = P.weight.empty() ? nullptr : m.upload(P.weight);
      D.delta = m.get_n<double>(G.nslots);
      if (h->opt.patch_assembly == VK_ASSEMBLY_MATRIX_FREE) {
        D.pe.nloc = H.nloc;
        D.pe.ncell_lower = H.ncell_lower;
        D.pe.cell_dofs = m.upload(H.cell_dofs);
        D.pe.kel = m.upload(H.kel);
        D.pe.cell_ptr = m.upload(H.patch_cell_ptr);
        D.pe.cells = m.upload(H.patch_cells);
      }
      if (h->opt.factor_prec == VK_PREC_F64E) D.r2 = m.get_n<float2>(H.ndof);
    }
  }
  h->nc = h->host[0].ndof;
  const int mdim = h->nc + 1;
  h->Cinv = m.get_n<double>(size_t(mdim) * mdim);
  const int nf = h->host[L - 1].ndof;
  h->kmax = h->opt.max_iterations;
  h->ldv = (int64_t(nf) + 31) / 32 * 32;
  h->V = m.get_n<double>(size_t(h->ldv) * (h->kmax + 1));
  h->Z = m.get_n<double>(size_t(h->ldv) * h->kmax);
  h->H = m.get_n<double>(size_t(h->kmax + 1) * h->kmax);
  h->cs = m.get_n<double>(h->kmax);
  h->sn = m.get_n<double>(h->kmax);
  h->g = m.get_n<double>(h->kmax + 1);
  h->hist = m.get_n<double>(h->kmax + 1);
  h->yv = m.get_n<double>(h->kmax);
  h->t2 = m.get_n<double>(h->kmax + 1);
  h->partial = m.get_n<double>(size_t(vk::gpu::kReduceBlocks) * (std::max(h->kmax, mdim) + 1));
  h->scal = m.get_n<double>(16);
  h->iflag = m.get_n<int>(16);
  h->bh = m.get_n<double>(nf);
  h->xh = m.get_n<double>(nf);
  h->vin = m.get_n<double>(nf);
  h->zbuf = m.get_n<double>(nf);
  h->wbuf = m.get_n<double>(nf);
  h->st = m.get_n<vk::gpu::FgState>(1);
  if (h->opt.batch_prec != VK_BATCH_NONE) allocate_batch(h);
}

// Finest-level patch applications are bracketed by CUDA events on their stream when timing is on.
void timed_apply(vk_hierarchy* h, int l, const double* r, cudaStream_t s) {
  DevLevel& D = h->lv[l];
  const bool t = h->time_apply && l == h->prob.nlevels - 1;
  if (t) h->tm_apply.begin(s);
  h->n_launch += vk::gpu::patch_apply(D.pat, r, D.r2, D.delta, s);
  if (t) h->tm_apply.end(s);
}

double device_dot(vk_hierarchy* h, const double* x, const double* y, int n, cudaStream_t s) {
  h->n_launch += vk::gpu::dot_partials(x, y, n, h->partial, s);
  h->n_launch += vk::gpu::finalize_sum(h->partial, vk::gpu::kReduceBlocks, h->scal, s);
  CK(cudaMemcpyAsync(h->h_scal, h->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return h->h_scal[0];
}

void vanka_apply(vk_hierarchy* h, int l, const double* r, double* z, cudaStream_t s) {
  DevLevel& D = h->lv[l];
  timed_apply(h, l, r, s);
  h->n_launch += vk::gpu::vanka_scatter(D.pat, D.ndof, D.dir, r, D.delta, 0, 1.0, 0.0, 0.0, z, nullptr, nullptr, s);
}

// nu Chebyshev steps on [lo*lam, hi*lam] (Sec. 3), preconditioned by additive Vanka (Algorithm 1);
// the Chebyshev coefficients follow the three-term recurrence (rho_k = 1/(2 sigma - rho_{k-1})).
void smooth(vk_hierarchy* h, int l, const double* b, double* x, bool zero_init, cudaStream_t s) {
  DevLevel& D = h->lv[l];
  const double lam = D.lam;
  const double emax = h->opt.cheb_hi * lam, emin = h->opt.cheb_lo * lam;
  const double theta = 0.5 * (emax + emin), delta = 0.5 * (emax - emin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  for (int step = 0; step < h->opt.sweeps; ++step) {
    const double* rr = b;
    if (!(step == 0 && zero_init)) {
      h->n_launch += vk::gpu::sell_residual(D.A, b, x, D.r, s);
      rr = D.r;
    }
    timed_apply(h, l, rr, s);
    int mode;
    double c1 = 0.0, c2 = 0.0;
    if (step == 0) {
      mode = zero_init ? 1 : 2;
    } else {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      c1 = rho_new * rho;
      c2 = 2.0 * rho_new / delta;
      rho = rho_new;
      mode = 3;
    }
    h->n_launch += vk::gpu::vanka_scatter(D.pat, D.ndof, D.dir, rr, D.delta, mode, theta, c1, c2, nullptr, D.d, x, s);
  }
}

void vcycle(vk_hierarchy* h, int l, const double* b, double* x, cudaStream_t s, bool count = true) {
  if (l == h->prob.nlevels - 1 && count) ++h->n_vcycle;
  if (l == 0) {
    h->n_launch += vk::gpu::dense_gemv(h->Cinv, h->nc, h->nc + 1, b, x, s);
    return;
  }
  DevLevel& D = h->lv[l];
  DevLevel& C = h->lv[l - 1];
  smooth(h, l, b, x, true, s);
  const bool t = h->time_apply && l == h->prob.nlevels - 1;
  if (t) h->tm_spmv.begin(s);
  h->n_launch += vk::gpu::sell_residual(D.A, b, x, D.r, s);
  if (t) h->tm_spmv.end(s);
  h->n_launch += vk::gpu::sell_restrict(D.R, C.dir, D.r, C.b, s);
  vcycle(h, l - 1, C.b, C.x, s, count);
  h->n_launch += vk::gpu::sell_prolong_add(D.P, C.x, x, s);
  smooth(h, l, b, x, false, s);
}

// "standard GMRES estimation" (Sec. 3) read as eig_steps Arnoldi steps (modified Gram-Schmidt) on
// M^{-1} A from a SplitMix64 start vector with Dirichlet entries zeroed and the pressure mean removed;
// lambda = largest real part of the Ritz values.  Breakdown: ||w_orth|| <= 1e-12 ||M^{-1} A v_j||.
double estimate_lambda(vk_hierarchy* h, int l, cudaStream_t s) {
  const vk::HostLevel& H = h->host[l];
  DevLevel& D = h->lv[l];
  const int n = H.ndof, steps = h->opt.eig_steps;
  std::vector<double> v0(n);
  for (int i = 0; i < n; ++i) v0[i] = H.dir[i] ? 0.0 : vk::splitmix_uniform_pm1(h->opt.eig_seed + uint64_t(l), i);
  double ps = 0.0;
  for (int i = H.n_u; i < n; ++i) ps += v0[i];
  const double mean = ps / H.n_p;
  for (int i = H.n_u; i < n; ++i) v0[i] -= mean;
  double nrm = 0.0;
  for (double v : v0) nrm += v * v;
  nrm = std::sqrt(nrm);
  for (double& v : v0) v /= nrm;
  if (steps + 1 > h->kmax + 1) raise(VK_ERR_ARG, "eig_steps exceeds the Krylov workspace");
  const int64_t ld = h->ldv;
  CK(cudaMemcpyAsync(h->V, v0.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  std::vector<double> Hm(size_t(steps + 1) * steps, 0.0);  // row-major (steps+1) x steps
  int m = steps;
  for (int j = 0; j < steps; ++j) {
    double* vj = h->V + ld * j;
    double* w = h->V + ld * (j + 1);
    h->n_launch += vk::gpu::sell_residual(D.A, nullptr, vj, D.t, s);
    vanka_apply(h, l, D.t, w, s);
    const double wnorm = std::sqrt(device_dot(h, w, w, n, s));
    for (int i = 0; i <= j; ++i) {
      const double hij = device_dot(h, h->V + ld * i, w, n, s);
      Hm[size_t(i) * steps + j] = hij;
      h->n_launch += vk::gpu::axpy(-hij, h->V + ld * i, w, n, s);
    }
    const double hn = std::sqrt(device_dot(h, w, w, n, s));
    Hm[size_t(j + 1) * steps + j] = hn;
    if (hn <= 1e-12 * wnorm) {
      m = j + 1;
      break;
    }
    h->n_launch += vk::gpu::divide(hn, w, n, s);
  }
  std::vector<double> sq(size_t(m) * m), re(m), im(m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) sq[size_t(i) * m + j] = Hm[size_t(i) * steps + j];
  if (vk::hessenberg_eigenvalues(m, sq.data(), re.data(), im.data()) != 0)
    raise(VK_ERR_INTERNAL, "Hessenberg QR did not converge on level " + std::to_string(l));
  return *std::max_element(re.begin(), re.end());
}

// Autotuner of the patch application: on every smoothed level, time each candidate launch shape
// (CUDA events on the setup stream, best of `reps` launches after one warm-up launch) on the level's
// own patches and keep the fastest.  Every shape gives bit-identical corrections, so the choice only
// changes speed.  opt.apply_schedule >= 0 forces that candidate instead (no timing).
void tune_patch_apply(vk_hierarchy* h, cudaStream_t s) {
  const auto cand = apply_candidates();
  const int L = h->prob.nlevels;
  h->tune.assign(L, TuneResult{});
  if (h->opt.apply_schedule >= int(cand.size())) raise(VK_ERR_ARG, "apply_schedule out of range");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  try {
    for (int l = 1; l < L; ++l) {
      DevLevel& D = h->lv[l];
      TuneResult& T = h->tune[l];
      if (h->opt.apply_schedule >= 0) {
        T.index = h->opt.apply_schedule;
      } else if (h->opt.autotune) {
        h->n_launch += vk::gpu::fill(D.t, 1.0, D.ndof, s);
        const int reps = 3;
        double best = 1e300;
        for (size_t i = 0; i < cand.size(); ++i) {
          h->n_launch += vk::gpu::patch_apply_sched(D.pat, cand[i], D.t, D.r2, D.delta, s);
          float t_best = 1e30f;
          for (int k = 0; k < reps; ++k) {
            CK(cudaEventRecord(e0, s));
            h->n_launch += vk::gpu::patch_apply_sched(D.pat, cand[i], D.t, D.r2, D.delta, s);
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            t_best = std::min(t_best, ms);
          }
          T.us[i] = 1e3 * t_best;
          if (T.us[i] < best) {
            best = T.us[i];
            T.index = int(i);
          }
        }
        CK(cudaGetLastError());
      }
      D.pat.sched = cand[T.index];
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
}

void setup_device(vk_hierarchy* h, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_device_mu);
  h->mem.stream = s;
  allocate_device(h);
  CK(cudaMallocHost(&h->h_flag, 4 * sizeof(int)));
  CK(cudaMallocHost(&h->h_scal, 4 * sizeof(double)));
  CK(cudaMallocHost(&h->h_par, sizeof(vk::gpu::FgState)));
  CK(cudaMallocHost(&h->h_res, sizeof(vk::gpu::FgState)));
  CK(cudaMallocHost(&h->h_hist, (h->kmax + 1) * sizeof(double)));
  CK(cudaStreamCreateWithFlags(&h->cap0, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&h->cap1, cudaStreamNonBlocking));
  CK(cudaMemsetAsync(h->iflag, 0, 16 * sizeof(int), s));
  const int L = h->prob.nlevels;
  {
    // patch matrices (gathered or assembled) and their inverses, timed with events on the setup stream
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
    for (int l = 1; l < L; ++l) {
      DevLevel& D = h->lv[l];
      const vk::gpu::PatchElems* pe = h->opt.patch_assembly == VK_ASSEMBLY_MATRIX_FREE ? &D.pe : nullptr;
      const int nl = vk::gpu::patch_factor(D.Acsr, D.pat, D.pat.prec, const_cast<void*>(D.pat.factors), h->iflag + l,
                                           s, pe);
      if (nl < 0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        raise(VK_ERR_ARG, "level " + std::to_string(l) + " has a patch larger than the factor kernel supports");
      }
      h->n_launch += nl;
    }
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    h->factor_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
  }
  // coarsest level: bordered inverse
  {
    DevLevel& C = h->lv[0];
    const int mdim = h->nc + 1;
    h->n_launch += vk::gpu::bordered_from_csr(C.Acsr, C.n_u, h->Cinv, s);
    int* perm = reinterpret_cast<int*>(h->partial);  // scratch: mdim ints, mdim+1 doubles after them
    double* fcol = h->partial + (mdim + 1) / 2 + 1;
    h->n_launch += vk::gpu::gauss_jordan_inverse(h->Cinv, mdim, perm, fcol, h->iflag + 14, h->iflag, s);
    CK(cudaGetLastError());
  }
  if (h->opt.batch_prec != VK_BATCH_NONE) {
    const bool half = h->opt.batch_prec == VK_BATCH_FP16;
    for (int l = 1; l < L; ++l) {
      DevLevel& D = h->lv[l];
      h->n_launch += vk::gpu::pack_mma(D.pat, static_cast<const double*>(D.pat.factors), D.foff16, D.frag, D.ascale,
                                       half, s);
      h->n_launch += vk::gpu::pack_tc(D.pat, D.tc, static_cast<const double*>(D.pat.factors), D.ascale, half, s);
    }
    const int64_t mm = int64_t(h->nc + 1) * (h->nc + 1);
    if (h->opt.batch_coarse_fp32) h->n_launch += vk::gpu::to_f32(h->Cinv, h->cinv_f, mm, s);
    CK(cudaMemsetAsync(h->tc_err, 0, 4 * sizeof(int), s));
    CK(cudaGetLastError());
  }
  std::vector<int> st(16);
  CK(cudaMemcpyAsync(st.data(), h->iflag, 16 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int l = 1; l < L; ++l)
    if (st[l] != 0)
      raise(VK_ERR_SINGULAR, "zero pivot in patch " + std::to_string(st[l] - 1) + " on level " + std::to_string(l));
  if (st[0] != 0) raise(VK_ERR_SINGULAR, "zero pivot in the coarse bordered matrix");
  {
    const vk::HostLevel& F = h->host[L - 1];
    double sn = 0.0, sn2 = 0.0;
    const int np = int(F.patch_ptr.size()) - 1;
    for (int p = 0; p < np; ++p) {
      const double n = F.patch_ptr[p + 1] - F.patch_ptr[p];
      sn += n;
      sn2 += n * n;
    }
    const double fsz = h->opt.factor_prec == VK_PREC_F32 ? 4.0 : 8.0;
    // algorithmic bytes of one sweep: the stored inverse entries, one 4-byte DoF index per slot, and
    // the residual read plus the correction read and written once per DoF
    h->apply_bytes = fsz * sn2 + 4.0 * sn + 24.0 * double(F.ndof);
    h->apply_flops = 2.0 * sn2;
    // residual SpMV r = b - A x: value + column index per stored nonzero; row index, b, x, r per row
    const double nnz = double(F.A.nnz()), nrow = double(F.ndof);
    h->spmv_bytes = 12.0 * nnz + 28.0 * nrow;
    // 16 right-hand sides in FP32: value + column per nonzero, row pointer, 16 x (b, x, r) per row
    h->bspmv_bytes = 8.0 * nnz + 4.0 * nrow + 3.0 * 64.0 * nrow;
    if (h->opt.batch_prec != VK_BATCH_NONE) {
      // compulsory traffic of one sweep: the 16-bit inverses as stored, the index tables as read,
      // every DoF's 16 FP32 residual values once (64 bytes) and 16 FP32 corrections per slot written
      double frag = 0.0, index = 0.0;
      if (h->opt.batch_engine == VK_ENGINE_MMA_SYNC) {
        for (int p = 0; p < np; ++p) frag += 16.0 * vk::gpu::frag_size(F.patch_ptr[p + 1] - F.patch_ptr[p]);
        index = 8.0 * sn + 20.0 * np;   // slot DoF and position; work, slot pointer, offset, scale
      } else {
        frag = h->lv[L - 1].tc_bytes;
        for (int c = 0; c < 3; ++c) {
          const double ng = h->lv[L - 1].tc.cls[c].ngroups, G = vk::gpu::kTcG[c], K = vk::gpu::kTcK[c];
          index += ng * (4.0 * G * K + 4.0 * 128 + 16.0 + 4.0 * G);   // gdof, gpos, gmeta, gscale
        }
      }
      h->bapply_bytes = frag + index + 64.0 * F.ndof + 64.0 * sn;
      h->bapply_flops = 2.0 * 16.0 * sn2;
    }
  }
  {
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    for (int l = 1; l < L; ++l) h->lv[l].pat.nsm = h->lv[l].tc.nsm = nsm;
  }
  tune_patch_apply(h, s);
  h->lambdas.assign(L, 0.0);
  for (int l = 1; l < L; ++l) {
    h->lambdas[l] = h->opt.lambdas ? h->opt.lambdas[l] : estimate_lambda(h, l, s);
    if (!(h->lambdas[l] > 0.0) || !std::isfinite(h->lambdas[l]))
      raise(VK_ERR_SINGULAR, "non-positive eigenvalue estimate on level " + std::to_string(l));
    h->lv[l].lam = h->lambdas[l];
  }
  CK(cudaStreamSynchronize(s));
}

void check_level(const vk_hierarchy* h, int level, int min_level = 0) {
  if (!h) raise(VK_ERR_ARG, "null hierarchy");
  if (level < min_level || level >= h->prob.nlevels) raise(VK_ERR_ARG, "level out of range");
}

void check_device(const vk_hierarchy* h) {
  if (!h) raise(VK_ERR_ARG, "null hierarchy");
  if (h->host_only) raise(VK_ERR_ARG, "host-only hierarchy: no device data");
}

int solve_graph(vk_hierarchy* h, const double* b, double* x, double rtol, int maxit, vk_solve_info* info,
                cudaStream_t s);

int solve_impl(vk_hierarchy* h, const double* b, double* x, double rtol, int maxit, vk_solve_info* info,
               cudaStream_t s) {
  check_device(h);
  if (!b || !x) raise(VK_ERR_ARG, "null vector");
  if (maxit < 1 || maxit > h->kmax) raise(VK_ERR_ARG, "maxit must be in 1..max_iterations");
  if (!(rtol >= 0.0)) raise(VK_ERR_ARG, "rtol must be >= 0");
  // graph path unless disabled, or unless per-launch kernel timing was requested (events cannot
  // bracket every iteration of a device-side loop)
  if (h->opt.use_graph && !h->time_apply) return solve_graph(h, b, x, rtol, maxit, info, s);
  const auto t0 = std::chrono::steady_clock::now();
  const int L = h->prob.nlevels;
  DevLevel& F = h->lv[L - 1];
  const int n = F.ndof;
  const int64_t ld = h->ldv;
  const int ldh = h->kmax + 1;
  // b_hat = b projected off the constant pressure; v_1 = b_hat / ||b_hat||
  h->n_launch += vk::gpu::copy(h->V, b, n, s);
  h->n_launch += vk::gpu::pressure_project(h->V, F.n_u, F.n_p, h->partial, h->scal + 1, s);
  const double beta = std::sqrt(device_dot(h, h->V, h->V, n, s));
  int status = VK_OK;
  int iters = 0;
  bool converged = false;
  std::vector<double> hist;
  if (!std::isfinite(beta)) raise(VK_ERR_NONFINITE, "right-hand side is not finite");
  if (beta == 0.0) {
    h->n_launch += vk::gpu::fill(x, 0.0, n, s);
    CK(cudaStreamSynchronize(s));
    converged = true;
    hist.assign(1, 0.0);
  } else {
    h->n_launch += vk::gpu::scale_copy(h->V, h->scal, h->V, n, s);   // v_1 = b_hat / beta (division)
    h->n_launch += vk::gpu::fill(h->g, 0.0, h->kmax + 1, s);
    CK(cudaMemcpyAsync(h->g, &beta, sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->hist, &beta, sizeof(double), cudaMemcpyHostToDevice, s));
    for (int j = 0; j < maxit; ++j) {
      double* vj = h->V + ld * j;
      double* zj = h->Z + ld * j;
      double* w = h->V + ld * (j + 1);
      double* hcol = h->H + int64_t(j) * ldh;
      vcycle(h, L - 1, vj, zj, s);
      h->n_launch += vk::gpu::pressure_project(zj, F.n_u, F.n_p, h->partial, h->scal + 1, s);
      h->n_launch += vk::gpu::sell_residual(F.A, nullptr, zj, w, s);
      // classical Gram-Schmidt, twice
      h->n_launch += vk::gpu::multi_dot_partials(h->V, ld, j + 1, w, n, h->partial, s);
      h->n_launch += vk::gpu::multi_finalize(h->partial, j + 1, hcol, nullptr, s);
      h->n_launch += vk::gpu::multi_axpy(h->V, ld, j + 1, hcol, w, n, s);
      h->n_launch += vk::gpu::multi_dot_partials(h->V, ld, j + 1, w, n, h->partial, s);
      h->n_launch += vk::gpu::multi_finalize(h->partial, j + 1, h->t2, hcol, s);
      h->n_launch += vk::gpu::multi_axpy(h->V, ld, j + 1, h->t2, w, n, s);
      h->n_launch += vk::gpu::dot_partials(w, w, n, h->partial, s);
      h->n_launch += vk::gpu::finalize_sum(h->partial, vk::gpu::kReduceBlocks, h->scal + 2, s);
      h->n_launch += vk::gpu::normalize(w, h->scal + 2, w, hcol + j + 1, n, s);
      h->n_launch += vk::gpu::givens_update(h->H, ldh, h->cs, h->sn, h->g, h->hist, j, rtol, h->iflag + 8, s);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(h->h_flag, h->iflag + 8, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      iters = j + 1;
      if (h->h_flag[1]) {
        status = VK_ERR_NONFINITE;
        g_err = "FGMRES residual estimate is not finite";
        break;
      }
      if (h->h_flag[0]) {
        converged = true;
        break;
      }
    }
    // y = H^{-1} g (upper triangular after the rotations), x = Z y
    const int m = iters;
    std::vector<double> Hh(size_t(ldh) * m), gh(m + 1), y(m);
    CK(cudaMemcpyAsync(Hh.data(), h->H, Hh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(gh.data(), h->g, (m + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    hist.assign(m + 1, 0.0);
    CK(cudaMemcpyAsync(hist.data(), h->hist, (m + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = m - 1; i >= 0; --i) {
      double acc = gh[i];
      for (int k = i + 1; k < m; ++k) acc -= Hh[size_t(k) * ldh + i] * y[k];
      y[i] = acc / Hh[size_t(i) * ldh + i];
    }
    CK(cudaMemcpyAsync(h->yv, y.data(), m * sizeof(double), cudaMemcpyHostToDevice, s));
    h->n_launch += vk::gpu::combine(h->Z, ld, m, h->yv, x, n, s);
  }
  // true residual of the projected system
  double true_res = 0.0;
  {
    h->n_launch += vk::gpu::copy(F.t, b, n, s);
    h->n_launch += vk::gpu::pressure_project(F.t, F.n_u, F.n_p, h->partial, h->scal + 1, s);
    h->n_launch += vk::gpu::sell_residual(F.A, F.t, x, F.r, s);
    true_res = std::sqrt(device_dot(h, F.r, F.r, n, s));
  }
  if (status == VK_OK && !converged) {
    status = VK_ERR_NOT_CONVERGED;
    g_err = "FGMRES did not reach rtol in maxit iterations";
  }
  if (info) {
    info->iterations = iters;
    info->converged = converged ? 1 : 0;
    info->res0 = beta;
    info->res_est = hist.empty() ? 0.0 : hist.back();
    info->true_res = true_res;
    if (info->history)
      for (size_t i = 0; i < hist.size(); ++i) info->history[i] = hist[i];
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

// One FGMRES solve as a CUDA graph: prologue (b_hat = projected bh, beta, v_1), a WHILE conditional
// node whose body is one iteration (V-cycle, projection, A z, CGS2, normalisation, Givens; the Givens
// kernel advances the device-side iteration counter and clears the condition on convergence or
// maxit), and an epilogue (back substitution, x = Z y into xh, true residual, copies of the state and
// history to pinned host memory).  Built once per hierarchy; only bh / xh are bound.
void build_graph_locked(vk_hierarchy* h);

void build_graph_attempt(vk_hierarchy* h, bool pdl);

// Captures the graph with programmatic dependent launch when the options ask for it; a driver that
// refuses such a capture gets the graph rebuilt with ordinary launches.
void build_graph(vk_hierarchy* h) {
  std::lock_guard<std::mutex> lock(g_device_mu);
  const bool want = h->opt.graph_pdl == 1;
  try {
    build_graph_attempt(h, want);
  } catch (...) {
    if (!want) throw;
    build_graph_attempt(h, false);
  }
}

void build_graph_attempt(vk_hierarchy* h, bool pdl) {
  vk::gpu::set_pdl(pdl);
  try {
    build_graph_locked(h);
    vk::gpu::set_pdl(false);
    h->graph_pdl = pdl ? 1 : 0;
  } catch (...) {
    vk::gpu::set_pdl(false);
    // leave no stream in capture mode and no half-built graph behind
    cudaStreamCaptureStatus st;
    for (cudaStream_t c : {h->cap1, h->cap0})
      if (c && cudaStreamIsCapturing(c, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(c, &g);
        if (g) cudaGraphDestroy(g);
      }
    cudaGetLastError();
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    throw;
  }
}

void build_graph_locked(vk_hierarchy* h) {
  const int L = h->prob.nlevels;
  DevLevel& F = h->lv[L - 1];
  const int n = F.ndof;
  const int64_t ld = h->ldv;
  const int ldh = h->kmax + 1;
  cudaStream_t c0 = h->cap0, c1 = h->cap1;
  const bool timing = h->time_apply;
  h->time_apply = false;
  const int64_t launches0 = h->n_launch;
  CK(cudaStreamBeginCapture(c0, cudaStreamCaptureModeRelaxed));
  h->n_launch += vk::gpu::copy(h->V, h->bh, n, c0);
  h->n_launch += vk::gpu::pressure_project(h->V, F.n_u, F.n_p, h->partial, h->scal + 1, c0);
  h->n_launch += vk::gpu::dot_partials(h->V, h->V, n, h->partial, c0);
  h->n_launch += vk::gpu::finalize_sum(h->partial, vk::gpu::kReduceBlocks, h->scal, c0);
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  CK(cudaStreamGetCaptureInfo(c0, &cst, nullptr, &g, &deps, nullptr, &ndeps));
  CK(cudaGraphConditionalHandleCreate(&h->cond, g, 0, 0));
  h->n_launch += vk::gpu::fg_init(h->scal, h->st, h->g, h->hist, h->kmax, h->cond, c0);
  h->n_launch += vk::gpu::fg_scale(h->V, h->st, n, h->vin, c0);
  h->g_pro = h->n_launch - launches0;
  CK(cudaStreamGetCaptureInfo(c0, &cst, nullptr, &g, &deps, nullptr, &ndeps));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h->cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  CK(cudaGraphAddNode(&cnode, g, deps, nullptr, ndeps, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(cudaStreamUpdateCaptureDependencies(c0, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  // loop body, captured straight into the conditional node's body graph
  const int64_t launches1 = h->n_launch;
  CK(cudaStreamBeginCaptureToGraph(c1, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  // vin holds V[j]: written by the prologue's scaling for j = 0, by the previous normalisation after
  vcycle(h, L - 1, h->vin, h->zbuf, c1, false);
  h->n_launch += vk::gpu::fg_project_put(h->zbuf, h->Z, ld, h->st, n, F.n_u, h->partial, h->scal + 1, c1);
  h->n_launch += vk::gpu::sell_residual(F.A, nullptr, h->zbuf, h->wbuf, c1);
  h->n_launch += vk::gpu::fg_cgs_pass(h->V, ld, h->st, h->wbuf, n, h->partial, h->H, ldh, h->t2, h->kmax, 0, c1);
  h->n_launch += vk::gpu::fg_cgs_pass(h->V, ld, h->st, h->wbuf, n, h->partial, h->H, ldh, h->t2, h->kmax, 1, c1);
  h->n_launch += vk::gpu::dot_partials(h->wbuf, h->wbuf, n, h->partial, c1);
  h->n_launch += vk::gpu::finalize_sum(h->partial, vk::gpu::kReduceBlocks, h->scal + 2, c1);
  h->n_launch += vk::gpu::fg_normalize(h->wbuf, h->scal + 2, h->V, ld, h->st, h->H, ldh, n, h->vin, c1);
  h->n_launch += vk::gpu::fg_givens(h->H, ldh, h->cs, h->sn, h->g, h->hist, h->st, h->cond, c1);
  cudaGraph_t body_out = nullptr;
  CK(cudaStreamEndCapture(c1, &body_out));
  h->g_body = h->n_launch - launches1;
  // epilogue
  const int64_t launches2 = h->n_launch;
  h->n_launch += vk::gpu::fg_solution(h->H, ldh, h->g, h->Z, ld, h->st, h->yv, h->xh, n, c0);
  h->n_launch += vk::gpu::copy(F.t, h->bh, n, c0);
  h->n_launch += vk::gpu::pressure_project(F.t, F.n_u, F.n_p, h->partial, h->scal + 1, c0);
  h->n_launch += vk::gpu::sell_residual(F.A, F.t, h->xh, F.r, c0);
  h->n_launch += vk::gpu::dot_partials(F.r, F.r, n, h->partial, c0);
  h->n_launch += vk::gpu::finalize_sum(h->partial, vk::gpu::kReduceBlocks, h->scal + 3, c0);
  h->n_launch += vk::gpu::fg_finish(h->st, h->scal + 3, c0);
  CK(cudaMemcpyAsync(h->h_res, h->st, sizeof(vk::gpu::FgState), cudaMemcpyDeviceToHost, c0));
  CK(cudaMemcpyAsync(h->h_hist, h->hist, (h->kmax + 1) * sizeof(double), cudaMemcpyDeviceToHost, c0));
  h->g_epi = h->n_launch - launches2;
  CK(cudaStreamEndCapture(c0, &h->graph));
  CK(cudaGraphInstantiate(&h->gexec, h->graph, 0));
  h->n_launch = launches0;
  h->time_apply = timing;
}

int solve_graph(vk_hierarchy* h, const double* b, double* x, double rtol, int maxit, vk_solve_info* info,
                cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!h->gexec) build_graph(h);
  const int n = h->lv.back().ndof;
  std::memset(h->h_par, 0, sizeof(vk::gpu::FgState));
  h->h_par->maxit = maxit;
  h->h_par->rtol = rtol;
  CK(cudaMemcpyAsync(h->st, h->h_par, sizeof(vk::gpu::FgState), cudaMemcpyHostToDevice, s));
  if (b != h->bh) CK(cudaMemcpyAsync(h->bh, b, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaGraphLaunch(h->gexec, s));
  if (x != h->xh) CK(cudaMemcpyAsync(x, h->xh, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  const vk::gpu::FgState r = *h->h_res;
  const int iters = r.j;
  h->n_launch += h->g_pro + int64_t(iters) * h->g_body + h->g_epi;
  h->n_vcycle += iters;
  int status = VK_OK;
  if (r.flags & 2) {
    status = iters == 0 ? VK_ERR_NONFINITE : VK_ERR_NONFINITE;
    g_err = iters == 0 ? "right-hand side is not finite" : "FGMRES residual estimate is not finite";
  } else if (!(r.flags & 1)) {
    status = VK_ERR_NOT_CONVERGED;
    g_err = "FGMRES did not reach rtol in maxit iterations";
  }
  if (info) {
    info->iterations = iters;
    info->converged = (r.flags & 1) ? 1 : 0;
    info->res0 = r.beta;
    info->res_est = h->h_hist[iters];
    info->true_res = r.true_res;
    if (info->history)
      for (int i = 0; i <= iters; ++i) info->history[i] = h->h_hist[i];
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

// ---- multi-right-hand-side solve ----------------------------------------------------------------
void smooth_b(vk_hierarchy* h, int l, const float* b, float* x, bool zero_init, cudaStream_t s) {
  DevLevel& D = h->lv[l];
  const bool half = h->opt.batch_prec == VK_BATCH_FP16;
  const double lam = D.lam;
  const double emax = h->opt.cheb_hi * lam, emin = h->opt.cheb_lo * lam;
  const double theta = 0.5 * (emax + emin), delta = 0.5 * (emax - emin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  for (int step = 0; step < h->opt.sweeps; ++step) {
    const float* rr = b;
    if (!(step == 0 && zero_init)) {
      h->n_launch += vk::gpu::mm_sell<float>(D.Ab, D.Ab.valf, 0, b, nullptr, x, D.rb, s);
      rr = D.rb;
    }
    const bool t = h->time_apply && l == h->prob.nlevels - 1;
    if (t) h->tm_apply.begin(s);
    if (h->opt.batch_engine == VK_ENGINE_MMA_SYNC)
      h->n_launch += vk::gpu::patch_apply_mma(D.pat, D.foff16, D.frag, D.ascale, half, D.mt_max, rr, D.delta_f, s);
    else
    {
      // test hook: the first finest-level sweep after setup withholds one bulk copy (see vk_options)
      const int skip = (h->expire_once && l == h->prob.nlevels - 1) ? 0 : -1;
      if (skip == 0) h->expire_once = false;
      h->n_launch += vk::gpu::patch_apply_tc(D.tc, half, rr, D.delta_f, h->tc_err, skip, s);
    }
    if (t) h->tm_apply.end(s);
    int mode;
    double c1 = 0.0, c2 = 0.0;
    if (step == 0) {
      mode = zero_init ? 1 : 2;
    } else {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      c1 = rho_new * rho;
      c2 = 2.0 * rho_new / delta;
      rho = rho_new;
      mode = 3;
    }
    h->n_launch += vk::gpu::scatter_mm(D.pat, D.ndof, D.dir, rr, D.delta_f, mode, float(theta), float(c1), float(c2),
                                       nullptr, D.db, x, s);
  }
}

void vcycle_b(vk_hierarchy* h, int l, const float* b, float* x, cudaStream_t s) {
  if (l == 0) {
    if (h->opt.batch_coarse_fp32) {
      h->n_launch += vk::gpu::coarse_mm(h->cinv_f, h->nc, h->nc + 1, b, x, s);
    } else {
      // the coarsest-level solve stays FP64: widen the FP32 right-hand sides, apply the FP64
      // bordered inverse, round the solution back for the FP32 V-cycle
      const int64_t len = int64_t(h->nc) * 16;
      h->n_launch += vk::gpu::to_f64(b, h->cb64, len, s);
      h->n_launch += vk::gpu::coarse_mm64(h->Cinv, h->nc, h->nc + 1, h->cb64, h->cx64, s);
      h->n_launch += vk::gpu::to_f32(h->cx64, x, len, s);
    }
    return;
  }
  DevLevel& D = h->lv[l];
  DevLevel& C = h->lv[l - 1];
  smooth_b(h, l, b, x, true, s);
  const bool t = h->time_apply && l == h->prob.nlevels - 1;
  if (t) h->tm_spmv.begin(s);
  h->n_launch += vk::gpu::mm_sell<float>(D.Ab, D.Ab.valf, 0, b, nullptr, x, D.rb, s);
  if (t) h->tm_spmv.end(s);
  h->n_launch += vk::gpu::mm_sell<float>(D.Rb, D.Rb.valf, 3, nullptr, C.dir, D.rb, C.bb, s);
  vcycle_b(h, l - 1, C.bb, C.xb, s);
  h->n_launch += vk::gpu::mm_sell<float>(D.Pb, D.Pb.valf, 2, x, nullptr, C.xb, x, s);
  smooth_b(h, l, b, x, false, s);
}

int solve_batch_impl(vk_hierarchy* h, int nrhs, const double* B, int64_t ldb, double* X, double rtol, int maxit,
                     vk_solve_info* infos, cudaStream_t s) {
  check_device(h);
  if (h->opt.batch_prec == VK_BATCH_NONE) raise(VK_ERR_ARG, "hierarchy built without batch_prec");
  constexpr int NR = 16;
  if (nrhs < 1 || nrhs > NR) raise(VK_ERR_ARG, "nrhs must be in 1..16");
  if (maxit < 1 || maxit > h->kb) raise(VK_ERR_ARG, "maxit must be in 1..batch_max_iterations");
  if (!B || !X) raise(VK_ERR_ARG, "null block vector");
  const auto t0 = std::chrono::steady_clock::now();
  const int L = h->prob.nlevels;
  DevLevel& F = h->lv[L - 1];
  const int n = F.ndof;
  if (ldb < n) raise(VK_ERR_ARG, "ldb < ndof");
  const int64_t ld = h->ldb;
  const int ldh = h->kb + 1;
  const int64_t hstride = int64_t(ldh) * h->kb;
  CK(cudaMemsetAsync(h->tc_err, 0, 4 * sizeof(int), s));
  // b_hat per column, beta, v_1
  h->n_launch += vk::gpu::gather_cols(B, ldb, nrhs, h->wb, n, s);
  h->n_launch += vk::gpu::project_mm(h->wb, F.n_u, F.n_p, h->partb, h->sqb + NR, s);
  h->n_launch += vk::gpu::mdot_mm(h->wb, 0, 1, h->wb, n, h->partb, h->sqb, nullptr, s);
  std::vector<double> sq(NR), beta(NR);
  CK(cudaMemcpyAsync(sq.data(), h->sqb, NR * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<int> active(NR, 0), zeros(NR, 0);
  std::vector<double> g0(size_t(NR) * ldh, 0.0);
  bool bad_rhs = false;
  for (int r = 0; r < NR; ++r) {
    beta[r] = std::sqrt(sq[r]);
    if (r < nrhs && !std::isfinite(beta[r])) bad_rhs = true;
    active[r] = (r < nrhs && beta[r] > 0.0 && std::isfinite(beta[r])) ? 1 : 0;
    g0[size_t(r) * ldh] = beta[r];
  }
  if (bad_rhs) raise(VK_ERR_NONFINITE, "a right-hand side is not finite");
  CK(cudaMemcpyAsync(h->activeb, active.data(), NR * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->itersb, zeros.data(), NR * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->nonfb, zeros.data(), NR * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->gb, g0.data(), g0.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->histb, g0.data(), g0.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  h->n_launch += vk::gpu::normalize_mm(h->wb, h->sqb, h->activeb, h->Vb, n, s);
  std::vector<int> act(NR);
  for (int j = 0; j < maxit && std::count(active.begin(), active.end(), 1) > 0; ++j) {
    double* vj = h->Vb + ld * j;
    double* zj = h->Zb + ld * j;
    h->n_launch += vk::gpu::to_f32(vj, F.bb, ld, s);
    vcycle_b(h, L - 1, F.bb, F.xb, s);
    ++h->n_vcycle;
    h->n_launch += vk::gpu::to_f64(F.xb, zj, ld, s);
    h->n_launch += vk::gpu::project_mm(zj, F.n_u, F.n_p, h->partb, h->sqb + NR, s);
    h->n_launch += vk::gpu::mm_sell<double>(F.Ab, F.Ab.vald, 1, nullptr, nullptr, zj, h->wb, s);
    h->n_launch += vk::gpu::mdot_mm(h->Vb, ld, j + 1, h->wb, n, h->partb, h->hcolb, nullptr, s);
    h->n_launch += vk::gpu::maxpy_mm(h->Vb, ld, j + 1, h->hcolb, h->wb, n, s);
    h->n_launch += vk::gpu::mdot_mm(h->Vb, ld, j + 1, h->wb, n, h->partb, h->t2b, h->hcolb, s);
    h->n_launch += vk::gpu::maxpy_mm(h->Vb, ld, j + 1, h->t2b, h->wb, n, s);
    h->n_launch += vk::gpu::mdot_mm(h->wb, 0, 1, h->wb, n, h->partb, h->sqb, nullptr, s);
    h->n_launch += vk::gpu::givens_mm(h->Hb, ldh, hstride, h->csb, h->snb, h->gb, h->histb, h->hcolb, h->sqb, j, rtol,
                                      h->activeb, h->itersb, h->nonfb, s);
    h->n_launch += vk::gpu::normalize_mm(h->wb, h->sqb, h->activeb, h->Vb + ld * (j + 1), n, s);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(act.data(), h->activeb, NR * sizeof(int), cudaMemcpyDeviceToHost, s));
    int tc_err_it = 0;
    CK(cudaMemcpyAsync(&tc_err_it, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (tc_err_it != 0) raise(VK_ERR_TIMEOUT, "a tensor-core patch solve's bounded wait expired");
    active = act;
  }
  // per-column solutions
  std::vector<int> iters(NR), nonf(NR);
  std::vector<double> Hh(size_t(NR) * hstride), gh(size_t(NR) * ldh), hist(size_t(NR) * ldh);
  CK(cudaMemcpyAsync(iters.data(), h->itersb, NR * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(nonf.data(), h->nonfb, NR * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(Hh.data(), h->Hb, Hh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(gh.data(), h->gb, gh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hist.data(), h->histb, hist.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  int tc_err = 0;
  CK(cudaMemcpyAsync(&tc_err, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (tc_err != 0) raise(VK_ERR_TIMEOUT, "a tensor-core patch solve's bounded wait expired");
  std::vector<double> y(size_t(NR) * ldh, 0.0);
  for (int r = 0; r < NR; ++r) {
    const int mr = iters[r];
    const double* Hr = Hh.data() + size_t(r) * hstride;
    for (int i = mr - 1; i >= 0; --i) {
      double acc = gh[size_t(r) * ldh + i];
      for (int k = i + 1; k < mr; ++k) acc -= Hr[size_t(k) * ldh + i] * y[size_t(r) * ldh + k];
      y[size_t(r) * ldh + i] = acc / Hr[size_t(i) * ldh + i];
    }
  }
  CK(cudaMemcpyAsync(h->yb, y.data(), y.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  h->n_launch += vk::gpu::combine_mm(h->Zb, ld, h->itersb, h->yb, ldh, h->xob, n, s);
  // true residuals of the projected systems
  h->n_launch += vk::gpu::gather_cols(B, ldb, nrhs, h->wb, n, s);
  h->n_launch += vk::gpu::project_mm(h->wb, F.n_u, F.n_p, h->partb, h->sqb + NR, s);
  h->n_launch += vk::gpu::mm_sell<double>(F.Ab, F.Ab.vald, 0, h->wb, nullptr, h->xob, h->Zb, s);
  h->n_launch += vk::gpu::mdot_mm(h->Zb, 0, 1, h->Zb, n, h->partb, h->sqb, nullptr, s);
  h->n_launch += vk::gpu::scatter_cols(h->xob, X, ldb, nrhs, n, s);
  CK(cudaMemcpyAsync(sq.data(), h->sqb, NR * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int status = VK_OK;
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int r = 0; r < nrhs; ++r) {
    const bool conv = beta[r] == 0.0 || (!nonf[r] && hist[size_t(r) * ldh + iters[r]] <= rtol * beta[r]);
    if (nonf[r]) status = VK_ERR_NONFINITE;
    else if (!conv && status == VK_OK) status = VK_ERR_NOT_CONVERGED;
    if (infos) {
      infos[r].iterations = iters[r];
      infos[r].converged = conv ? 1 : 0;
      infos[r].res0 = beta[r];
      infos[r].res_est = hist[size_t(r) * ldh + iters[r]];
      infos[r].true_res = std::sqrt(sq[r]);
      infos[r].solve_ms = ms;
    }
  }
  if (status == VK_ERR_NONFINITE) g_err = "a column's residual estimate is not finite";
  if (status == VK_ERR_NOT_CONVERGED) g_err = "a column did not reach rtol in maxit iterations";
  return status;
}

const vk::HostCsr& pick_csr(const vk_hierarchy* h, int level, int which) {
  const vk::HostLevel& L = h->host[level];
  if (which == VK_CSR_A) return L.A;
  if (level < 1) raise(VK_ERR_ARG, "P and R exist from level 1");
  if (which == VK_CSR_P) return L.P;
  if (which == VK_CSR_R) return L.R;
  raise(VK_ERR_ARG, "unknown matrix");
}

}  // namespace

extern "C" {

void vk_default_options(vk_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->sweeps = 1;
  o->weights = VK_WEIGHTS_PLAIN;
  o->cheb_lo = 0.25;
  o->cheb_hi = 1.1;
  o->eig_steps = 10;
  o->eig_seed = 0x5EED;
  o->lambdas = nullptr;
  o->factor_prec = VK_PREC_F64;
  o->use_graph = 1;
  o->host_threads = 0;
  o->host_only = 0;
  o->max_iterations = 100;
  o->batch_prec = VK_BATCH_NONE;
  o->batch_max_iterations = 60;
  o->autotune = 1;
  o->apply_schedule = -1;
  o->batch_engine = VK_ENGINE_TCGEN05;
  o->spmv_warps = 48;
  o->test_singular_patch = -1;
  o->graph_pdl = 0;
}

int vk_check_problem(const vk_problem* p, const vk_options* o) {
  return guard([&] {
    validate(p, o);
    return VK_OK;
  });
}

const char* vk_last_error(void) { return g_err.c_str(); }

int vk_setup(const vk_problem* p, const vk_options* o, const vk_allocator* alloc, void* stream,
             vk_hierarchy** out) {
  return guard([&] {
    if (!out) raise(VK_ERR_ARG, "null output pointer");
    *out = nullptr;
    validate(p, o);
    auto h = std::make_unique<vk_hierarchy>();
    h->prob = *p;
    h->opt = *o;
    h->opt.lambdas = nullptr;
    h->host_only = o->host_only != 0;
    h->expire_once = o->test_expire_wait != 0;
    if (alloc && alloc->alloc && alloc->release) {
      h->mem.user = *alloc;
      h->mem.custom = true;
    }
    const auto t_setup = std::chrono::steady_clock::now();
    build_host(h.get());
    if (!h->host_only) {
      vk_options tmp = h->opt;
      h->opt.lambdas = o->lambdas;
      try {
        setup_device(h.get(), static_cast<cudaStream_t>(stream));
      } catch (...) {
        cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        h->mem.release_all();
        if (h->h_flag) cudaFreeHost(h->h_flag);
        if (h->h_scal) cudaFreeHost(h->h_scal);
        throw;
      }
      h->opt = tmp;
    }
    h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_setup).count();
    *out = h.release();
    return VK_OK;
  });
}

void vk_destroy(vk_hierarchy* h) {
  if (!h) return;
  std::lock_guard<std::mutex> lock(g_device_mu);
  if (!h->host_only) {
    cudaDeviceSynchronize();
    h->mem.release_all();
    if (h->h_flag) cudaFreeHost(h->h_flag);
    if (h->h_scal) cudaFreeHost(h->h_scal);
  }
  delete h;
}

int vk_footprint(const vk_problem* p, const vk_options* o, size_t* device_bytes) {
  return guard([&] {
    validate(p, o);
    if (!device_bytes) raise(VK_ERR_ARG, "null output");
    vk_hierarchy h;
    h.prob = *p;
    h.opt = *o;
    build_host(&h);
    h.mem.counting_only = true;
    allocate_device(&h);
    *device_bytes = h.mem.total;
    return VK_OK;
  });
}

int vk_device_bytes(const vk_hierarchy* h, size_t* bytes) {
  return guard([&] {
    if (!h || !bytes) raise(VK_ERR_ARG, "null argument");
    *bytes = h->mem.total;
    return VK_OK;
  });
}

int vk_level_info(const vk_hierarchy* h, int level, int32_t* ndof, int32_t* n_u, int64_t* nnz, int32_t* npatch,
                  int64_t* nslots) {
  return guard([&] {
    check_level(h, level);
    const vk::HostLevel& L = h->host[level];
    if (ndof) *ndof = L.ndof;
    if (n_u) *n_u = L.n_u;
    if (nnz) *nnz = L.A.nnz();
    if (npatch) *npatch = L.patch_ptr.empty() ? 0 : int32_t(L.patch_ptr.size() - 1);
    if (nslots) *nslots = int64_t(L.patch_dofs.size());
    return VK_OK;
  });
}

int vk_lambda(const vk_hierarchy* h, int level, double* lambda) {
  return guard([&] {
    check_level(h, level, 1);
    check_device(h);
    if (!lambda) raise(VK_ERR_ARG, "null output");
    *lambda = h->lambdas[level];
    return VK_OK;
  });
}

int vk_apply_schedule(const vk_hierarchy* h, int level, int32_t* split, int32_t* threads, int32_t* per_sm,
                      int32_t* index, double* cand_us, int32_t* ncand) {
  return guard([&] {
    check_level(h, level, 1);
    check_device(h);
    const auto cand = apply_candidates();
    const TuneResult& T = h->tune[level];
    const vk::gpu::ApplySched& sc = h->lv[level].pat.sched;
    if (split) *split = sc.split;
    if (threads) *threads = sc.threads;
    if (per_sm) *per_sm = sc.per_sm;
    if (index) *index = T.index;
    if (ncand) *ncand = int32_t(cand.size());
    if (cand_us)
      for (size_t i = 0; i < cand.size(); ++i) cand_us[i] = T.us[i];
    return VK_OK;
  });
}

int vk_residual(vk_hierarchy* h, int level, const double* b, const double* x, double* r, void* stream) {
  return guard([&] {
    check_level(h, level);
    check_device(h);
    if (!b || !x || !r) raise(VK_ERR_ARG, "null vector");
    h->n_launch += vk::gpu::sell_residual(h->lv[level].A, b, x, r, static_cast<cudaStream_t>(stream));
    CK(cudaGetLastError());
    return VK_OK;
  });
}

int vk_vanka(vk_hierarchy* h, int level, const double* r, double* z, void* stream) {
  return guard([&] {
    check_level(h, level, 1);
    check_device(h);
    if (!r || !z || r == z) raise(VK_ERR_ARG, "null or aliased vectors");
    vanka_apply(h, level, r, z, static_cast<cudaStream_t>(stream));
    CK(cudaGetLastError());
    return VK_OK;
  });
}

int vk_smooth(vk_hierarchy* h, int level, const double* b, double* x, int zero_init, void* stream) {
  return guard([&] {
    check_level(h, level, 1);
    check_device(h);
    if (!b || !x || b == x) raise(VK_ERR_ARG, "null or aliased vectors");
    smooth(h, level, b, x, zero_init != 0, static_cast<cudaStream_t>(stream));
    CK(cudaGetLastError());
    return VK_OK;
  });
}

int vk_restrict(vk_hierarchy* h, int fine_level, const double* r_fine, double* r_coarse, void* stream) {
  return guard([&] {
    check_level(h, fine_level, 1);
    check_device(h);
    if (!r_fine || !r_coarse) raise(VK_ERR_ARG, "null vector");
    h->n_launch += vk::gpu::sell_restrict(h->lv[fine_level].R, h->lv[fine_level - 1].dir, r_fine, r_coarse,
                                          static_cast<cudaStream_t>(stream));
    CK(cudaGetLastError());
    return VK_OK;
  });
}

int vk_prolong(vk_hierarchy* h, int fine_level, const double* e_coarse, double* x_fine, void* stream) {
  return guard([&] {
    check_level(h, fine_level, 1);
    check_device(h);
    if (!e_coarse || !x_fine) raise(VK_ERR_ARG, "null vector");
    h->n_launch += vk::gpu::sell_prolong_add(h->lv[fine_level].P, e_coarse, x_fine, static_cast<cudaStream_t>(stream));
    CK(cudaGetLastError());
    return VK_OK;
  });
}

int vk_coarse_solve(vk_hierarchy* h, const double* b, double* x, void* stream) {
  return guard([&] {
    check_device(h);
    if (!b || !x) raise(VK_ERR_ARG, "null vector");
    h->n_launch += vk::gpu::dense_gemv(h->Cinv, h->nc, h->nc + 1, b, x, static_cast<cudaStream_t>(stream));
    CK(cudaGetLastError());
    return VK_OK;
  });
}

int vk_vcycle(vk_hierarchy* h, const double* b, double* x, void* stream) {
  return guard([&] {
    check_device(h);
    if (!b || !x || b == x) raise(VK_ERR_ARG, "null or aliased vectors");
    vcycle(h, h->prob.nlevels - 1, b, x, static_cast<cudaStream_t>(stream));
    CK(cudaGetLastError());
    return VK_OK;
  });
}

int vk_solve(vk_hierarchy* h, const double* b, double* x, double rtol, int maxit, vk_solve_info* info,
             void* stream) {
  return guard([&] { return solve_impl(h, b, x, rtol, maxit, info, static_cast<cudaStream_t>(stream)); });
}

int vk_solve_batch(vk_hierarchy* h, int nrhs, const double* B, int64_t ldb, double* X, double rtol, int maxit,
                   vk_solve_info* infos, void* stream) {
  return guard([&] { return solve_batch_impl(h, nrhs, B, ldb, X, rtol, maxit, infos, static_cast<cudaStream_t>(stream)); });
}

int vk_solve_host(vk_hierarchy* h, const double* b_host, double* x_host, double rtol, int maxit,
                  vk_solve_info* info, void* stream) {
  return guard([&] {
    check_device(h);
    if (!b_host || !x_host) raise(VK_ERR_ARG, "null vector");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = h->lv.back().ndof;
    const auto t0 = std::chrono::steady_clock::now();
    CK(cudaMemcpyAsync(h->bh, b_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
    int st = solve_impl(h, h->bh, h->xh, rtol, maxit, info, s);
    if (st != VK_OK && st != VK_ERR_NOT_CONVERGED) return st;
    CK(cudaMemcpyAsync(x_host, h->xh, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (info)
      info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return st;
  });
}

int vk_csr_dims(const vk_hierarchy* h, int level, int which, int32_t* nrows, int32_t* ncols, int64_t* nnz) {
  return guard([&] {
    check_level(h, level);
    const vk::HostCsr& A = pick_csr(h, level, which);
    if (nrows) *nrows = A.nrows;
    if (ncols) *ncols = A.ncols;
    if (nnz) *nnz = A.nnz();
    return VK_OK;
  });
}

int vk_export_csr(const vk_hierarchy* h, int level, int which, int32_t* ptr, int32_t* col, double* val) {
  return guard([&] {
    check_level(h, level);
    const vk::HostCsr& A = pick_csr(h, level, which);
    if (ptr) std::copy(A.ptr.begin(), A.ptr.end(), ptr);
    if (col) std::copy(A.col.begin(), A.col.end(), col);
    if (val) std::copy(A.val.begin(), A.val.end(), val);
    return VK_OK;
  });
}

int vk_export_patches(const vk_hierarchy* h, int level, int32_t* ptr, int32_t* dofs, int8_t* kind) {
  return guard([&] {
    check_level(h, level, 1);
    const vk::HostLevel& L = h->host[level];
    if (ptr) std::copy(L.patch_ptr.begin(), L.patch_ptr.end(), ptr);
    if (dofs) std::copy(L.patch_dofs.begin(), L.patch_dofs.end(), dofs);
    if (kind) std::copy(L.patch_kind.begin(), L.patch_kind.end(), kind);
    return VK_OK;
  });
}

int vk_ndof(const vk_hierarchy* h, int level, int64_t* n_u, int64_t* n_p) {
  return guard([&] {
    check_level(h, level);
    const vk::HostLevel& L = h->host[level];
    if (n_u) *n_u = L.n_u;
    if (n_p) *n_p = L.n_p;
    return VK_OK;
  });
}

int vk_export_dof_coords(const vk_hierarchy* h, int level, double* xy, int8_t* kind) {
  return guard([&] {
    check_level(h, level);
    if (!xy && !kind) raise(VK_ERR_ARG, "null outputs");
    const vk::HostLevel& L = h->host[level];
    if (L.cell == 2) {
      vk::bdm_dof_coords(L, xy, kind);
      return VK_OK;
    }
    const int nv = L.nv1, np = L.np1, kN = L.k * L.N, k1N = (L.k - 1) * L.N;
    for (int d = 0; d < L.ndof; ++d) {
      double x, y;
      int8_t c;
      if (d < L.n_u) {
        const int node = d / 2;
        x = double(node % nv) / kN;
        y = double(node / nv) / kN;
        c = int8_t(d & 1);
      } else {
        const int q = d - L.n_u;
        x = double(q % np) / k1N;
        y = double(q / np) / k1N;
        c = 2;
      }
      if (xy) {
        xy[2 * int64_t(d)] = x;
        xy[2 * int64_t(d) + 1] = y;
      }
      if (kind) kind[d] = c;
    }
    return VK_OK;
  });
}

int vk_export_dirichlet(const vk_hierarchy* h, int level, uint8_t* flags) {
  return guard([&] {
    check_level(h, level);
    if (!flags) raise(VK_ERR_ARG, "null output");
    const vk::HostLevel& L = h->host[level];
    std::copy(L.dir.begin(), L.dir.end(), flags);
    return VK_OK;
  });
}

int vk_stats_reset(vk_hierarchy* h, int time_kernels) {
  return guard([&] {
    check_device(h);
    h->n_launch = 0;
    h->n_vcycle = 0;
    h->tm_apply.used = 0;
    h->tm_spmv.used = 0;
    h->time_apply = time_kernels != 0;
    return VK_OK;
  });
}

int vk_stats_read(vk_hierarchy* h, vk_stats* out) {
  return guard([&] {
    check_device(h);
    if (!out) raise(VK_ERR_ARG, "null output");
    out->launches = h->n_launch;
    out->vcycles = h->n_vcycle;
    out->apply_launches = h->tm_apply.count();
    out->apply_ms = h->tm_apply.total_ms();
    out->apply_bytes = h->apply_bytes;
    out->apply_flops = h->apply_flops;
    out->batch_apply_bytes = h->bapply_bytes;
    out->batch_apply_flops = h->bapply_flops;
    out->spmv_launches = h->tm_spmv.count();
    out->spmv_ms = h->tm_spmv.total_ms();
    out->spmv_bytes = h->spmv_bytes;
    out->batch_spmv_bytes = h->bspmv_bytes;
    out->setup_factor_ms = h->factor_ms;
    out->setup_ms = h->setup_ms;
    out->graph_pdl = h->graph_pdl;
    return VK_OK;
  });
}

int vk_manufactured_rhs(const vk_hierarchy* h, double* b_host) {
  return guard([&] {
    if (!h || !b_host) raise(VK_ERR_ARG, "null argument");
    std::vector<double> b;
    if (h->prob.cell == VK_CELL_QUAD)
      vk::manufactured_rhs_quad(h->host.back(), h->prob.nu, b);
    else if (h->prob.cell == VK_CELL_BDM)
      vk::manufactured_rhs_bdm(h->host.back(), h->prob.nu, b);
    else
      vk::manufactured_rhs(h->host.back(), h->prob.nu, b);
    std::copy(b.begin(), b.end(), b_host);
    return VK_OK;
  });
}

int vk_errors(vk_hierarchy* h, const double* x, double* errs, void* stream) {
  return guard([&] {
    check_device(h);
    if (!x || !errs) raise(VK_ERR_ARG, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const vk::HostLevel& F = h->host.back();
    const bool quadc = h->prob.cell == VK_CELL_QUAD, bdmc = h->prob.cell == VK_CELL_BDM;
    std::vector<int> cv, cp;
    std::vector<double> xi, eta, w, phi, dxi, deta, psi, sg;
    if (bdmc) {
      vk::bdm_error_data(F, F.k + 6, cv, sg, cp, xi, eta, w, phi, dxi, psi);
      deta.assign(1, 0.0);
    } else if (quadc) {
      vk::cell_maps_quad(F.N, F.k, cv, cp);
      vk::reference_tables_quad(F.k, F.k + 6, xi, eta, w, phi, dxi, deta, psi);
    } else {
      vk::cell_maps(F.N, F.k, cv, cp);
      vk::reference_tables(F.k, F.k + 6, xi, eta, w, phi, dxi, deta, psi);
    }
    std::vector<void*> bufs;
    auto up = [&](const auto& v) {
      using T = typename std::decay_t<decltype(v)>::value_type;
      void* p = nullptr;
      CK(cudaMalloc(&p, std::max<size_t>(1, v.size()) * sizeof(T)));
      bufs.push_back(p);
      CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
      return static_cast<const T*>(p);
    };
    double sums[7] = {};
    try {
      vk::gpu::FemErrArgs a;
      a.N = F.N;
      a.quad = quadc ? 1 : 0;
      a.bdm = bdmc ? 1 : 0;
      a.nb = bdmc ? (F.k + 1) * (F.k + 2) : quadc ? (F.k + 1) * (F.k + 1) : (F.k + 1) * (F.k + 2) / 2;
      a.nq = quadc ? F.k * F.k : F.k * (F.k + 1) / 2;
      a.Q = int(w.size());
      a.n_u = F.n_u;
      a.h = 1.0 / F.N;
      a.cv = up(cv);
      a.cp = up(cp);
      a.xi = up(xi);
      a.eta = up(eta);
      a.w = up(w);
      a.phi = up(phi);
      a.dxi = up(dxi);
      a.deta = up(deta);
      a.psi = up(psi);
      if (bdmc) a.sg = up(sg);
      a.x = x;
      std::vector<double> zeros(1024 * 7 + 7, 0.0);
      double* part = const_cast<double*>(up(zeros));
      h->n_launch += vk::gpu::fem_error_sums(a, part, part + 1024 * 7, s);
      CK(cudaMemcpyAsync(sums, part + 1024 * 7, 7 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    } catch (...) {
      cudaStreamSynchronize(s);
      for (void* p : bufs) cudaFree(p);
      throw;
    }
    for (void* p : bufs) cudaFree(p);
    const double mean = sums[4] / sums[6];
    errs[0] = std::sqrt((sums[0] + sums[2]) / (sums[1] + sums[3]));
    errs[1] = std::sqrt(sums[0] / sums[1]);
    errs[2] = std::sqrt(std::max(sums[5] - 2.0 * mean * sums[4] + mean * mean * sums[6], 0.0));
    return VK_OK;
  });
}

int vk_measure_fma_rate(int precision, void* stream, double* tflops) {
  return guard([&] {
    if (!tflops || (precision != 0 && precision != 1)) raise(VK_ERR_ARG, "bad arguments");
    std::lock_guard<std::mutex> lock(g_device_mu);
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    void* scratch = nullptr;
    CK(cudaMalloc(&scratch, size_t(nsm) * 8 * 256 * 8));
    const double t = vk::gpu::fma_rate_tflops(precision == 0, scratch, static_cast<cudaStream_t>(stream));
    cudaFree(scratch);
    if (!(t > 0.0)) raise(VK_ERR_CUDA, "FMA-rate probe failed");
    *tflops = t;
    return VK_OK;
  });
}

int vk_hessenberg_eigenvalues(int m, const double* H, double* re, double* im) {
  return guard([&] {
    if (m < 1 || !H || !re || !im) raise(VK_ERR_ARG, "bad arguments");
    if (vk::hessenberg_eigenvalues(m, H, re, im) != 0) raise(VK_ERR_INTERNAL, "QR iteration did not converge");
    return VK_OK;
  });
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Allocation-free additive Vanka application.  Some callers cannot allocate device memory at the
// point where they need a relaxation sweep: a process whose device memory is fully reserved up front
// by another allocator (a pool that would fail or evict), or a latency-critical thread that must not
// hit the device-wide synchronisation cudaMalloc / cudaFree can imply.  vk_vanka keeps its per-slot
// corrections in a buffer the hierarchy allocated at setup; this variant keeps them instead in one
// fixed file-scope device array, so the call itself allocates nothing.
namespace {

constexpr int64_t kNoAllocMaxSlots = int64_t(1) << 20;  // 8 MiB of FP64 corrections per device
static __device__ __align__(256) double g_noalloc_delta[kNoAllocMaxSlots];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {};  // per device: address of g_noalloc_delta, set once

// Host code cannot use g_noalloc_delta directly (on the host it names a stand-in, not device
// memory): look its device address up once per device, with that device current.
double* noalloc_scratch() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) raise(VK_ERR_CUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_delta);
    if (e != cudaSuccess || !p)
      raise(VK_ERR_CUDA, std::string("cudaGetSymbolAddress(noalloc scratch): ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" int vk_vanka_noalloc(vk_hierarchy* h, int level, const double* r, double* z, void* stream) {
  return guard([&] {
    check_level(h, level, 1);
    check_device(h);
    if (!r || !z || r == z) raise(VK_ERR_ARG, "null or aliased vectors");
    DevLevel& D = h->lv[level];
    if (D.pat.nslots > kNoAllocMaxSlots)
      raise(VK_ERR_ARG, "level " + std::to_string(level) + " has " + std::to_string(D.pat.nslots) +
                            " patch slots; vk_vanka_noalloc supports at most " + std::to_string(kNoAllocMaxSlots));
    double* delta = noalloc_scratch();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // every slot is written by the patch solves before the sum reads it: nothing to clear
    h->n_launch += vk::gpu::patch_apply(D.pat, r, D.r2, delta, s);
    h->n_launch += vk::gpu::vanka_scatter(D.pat, D.ndof, D.dir, r, delta, 0, 1.0, 0.0, 0.0, z, nullptr, nullptr, s);
    CK(cudaGetLastError());
    return VK_OK;
  });
}

// ------------------------------------------------------------------------------------------------
// Group solve (vk_group_*): several independent FGMRES solves advanced together, one launch per stage
// over every active member.  Each member keeps its FGMRES state in its own hierarchy's workspace and
// runs exactly the host-driven loop of solve_impl, with every single-member launch replaced by the
// group launch of the same kernel body.
namespace {

struct GroupMember {
  vk_hierarchy* h = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  double rtol = 0.0, beta = 0.0, true_res = 0.0;
  int maxit = 0, j = 0, status = VK_OK;
  bool used = false, active = false, converged = false;
  std::vector<double> hist;
  std::chrono::steady_clock::time_point t0;
};

// one member's level in a group V-cycle, matched from the finest level down
struct GLevel {
  vk_hierarchy* h;
  int l;
  const double* b;
  double* x;
};

vk::gpu::GroupPatch group_patch(const DevLevel& D) {
  vk::gpu::GroupPatch g;
  g.work = D.pat.work;
  g.slot_ptr = D.pat.slot_ptr;
  g.slot_dofs = D.pat.slot_dofs;
  g.foff = D.pat.foff;
  g.factors = D.pat.factors;
  g.slot_pos = D.pat.slot_pos;
  g.dof_ptr = D.pat.dof_ptr;
  g.weight = D.pat.weight;
  g.dir = D.dir;
  g.sym = D.pat.sym;
  g.ndof = D.ndof;
  return g;
}

// group SpMV over the members' level matrices: which = 0 (A), 1 (P), 2 (R)
int64_t group_sell(const std::vector<GLevel>& ms, int which, int mode, const std::vector<const double*>& b,
                   const std::vector<const uint8_t*>& mask, const std::vector<const double*>& x,
                   const std::vector<double*>& y, cudaStream_t s) {
  vk::gpu::GroupSpmvArgs a;
  a.count = int(ms.size());
  for (int m = 0; m < a.count; ++m) {
    const DevLevel& D = ms[m].h->lv[ms[m].l];
    a.A[m] = which == 0 ? D.A : which == 1 ? D.P : D.R;
    a.prefix[m + 1] = a.prefix[m] + a.A[m].nslices;
    a.b[m] = b[m];
    a.mask[m] = mask[m];
    a.x[m] = x[m];
    a.y[m] = y[m];
  }
  return vk::gpu::group_spmv(mode, a, s);
}

// nu Chebyshev steps of every member's level (the arithmetic of smooth())
int64_t group_smooth(const std::vector<GLevel>& ms, bool zero_init, cudaStream_t s) {
  int64_t launches = 0;
  const int cnt = int(ms.size());
  const vk_options& o = ms[0].h->opt;
  std::vector<double> theta(cnt), delta(cnt), sigma(cnt), rho(cnt);
  for (int m = 0; m < cnt; ++m) {
    const double lam = ms[m].h->lv[ms[m].l].lam;
    const double emax = o.cheb_hi * lam, emin = o.cheb_lo * lam;
    theta[m] = 0.5 * (emax + emin);
    delta[m] = 0.5 * (emax - emin);
    sigma[m] = theta[m] / delta[m];
    rho[m] = 1.0 / sigma[m];
  }
  for (int step = 0; step < o.sweeps; ++step) {
    std::vector<const double*> rr(cnt);
    if (!(step == 0 && zero_init)) {
      std::vector<const double*> b(cnt), x(cnt), none(cnt, nullptr);
      std::vector<const uint8_t*> nomask(cnt, nullptr);
      std::vector<double*> r(cnt);
      for (int m = 0; m < cnt; ++m) {
        DevLevel& D = ms[m].h->lv[ms[m].l];
        b[m] = ms[m].b;
        x[m] = ms[m].x;
        r[m] = D.r;
        rr[m] = D.r;
      }
      launches += group_sell(ms, 0, 0, b, nomask, x, r, s);
    } else {
      for (int m = 0; m < cnt; ++m) rr[m] = ms[m].b;
    }
    vk::gpu::GroupApplyArgs ap;
    vk::gpu::GroupScatterArgs sc;
    ap.count = sc.count = cnt;
    ap.prec = sc.prec = ms[0].h->opt.factor_prec;
    int mode = 0;
    for (int m = 0; m < cnt; ++m) {
      DevLevel& D = ms[m].h->lv[ms[m].l];
      ap.P[m] = sc.P[m] = group_patch(D);
      ap.prefix[m + 1] = ap.prefix[m] + D.pat.npatch;
      ap.dprefix[m + 1] = ap.dprefix[m] + D.ndof;
      ap.nb_max = std::max(ap.nb_max, D.pat.nb_max);
      ap.r[m] = rr[m];
      ap.r2[m] = D.r2;
      ap.delta[m] = D.delta;
      sc.prefix[m + 1] = sc.prefix[m] + D.ndof;
      sc.r[m] = rr[m];
      sc.delta[m] = D.delta;
      sc.theta[m] = theta[m];
      sc.d[m] = D.d;
      sc.x[m] = ms[m].x;
      if (step == 0) {
        mode = zero_init ? 1 : 2;
      } else {
        const double rho_new = 1.0 / (2.0 * sigma[m] - rho[m]);
        sc.c1[m] = rho_new * rho[m];
        sc.c2[m] = 2.0 * rho_new / delta[m];
        rho[m] = rho_new;
        mode = 3;
      }
    }
    sc.mode = mode;
    launches += vk::gpu::group_patch_apply(ap, s);
    launches += vk::gpu::group_vanka_scatter(sc, s);
  }
  return launches;
}

// V(nu, nu) cycle of every member from its level ms[m].l down (the arithmetic of vcycle()).
int64_t group_vcycle(const std::vector<GLevel>& ms, cudaStream_t s) {
  int64_t launches = 0;
  std::vector<GLevel> coarse, rest;
  for (const GLevel& g : ms) (g.l == 0 ? coarse : rest).push_back(g);
  if (!coarse.empty()) {
    vk::gpu::GroupGemvArgs a;
    a.count = int(coarse.size());
    for (int m = 0; m < a.count; ++m) {
      vk_hierarchy* h = coarse[m].h;
      a.Minv[m] = h->Cinv;
      a.n[m] = h->nc;
      a.ld[m] = h->nc + 1;
      a.b[m] = coarse[m].b;
      a.x[m] = coarse[m].x;
      a.prefix[m + 1] = a.prefix[m] + h->nc;
    }
    launches += vk::gpu::group_dense_gemv(a, s);
  }
  if (rest.empty()) return launches;
  const int cnt = int(rest.size());
  launches += group_smooth(rest, true, s);
  std::vector<const double*> b(cnt), x(cnt), r(cnt), cx(cnt);
  std::vector<double*> rw(cnt), cb(cnt), xw(cnt);
  std::vector<const uint8_t*> nomask(cnt, nullptr), cdir(cnt);
  std::vector<GLevel> down(cnt);
  for (int m = 0; m < cnt; ++m) {
    DevLevel& D = rest[m].h->lv[rest[m].l];
    DevLevel& C = rest[m].h->lv[rest[m].l - 1];
    b[m] = rest[m].b;
    x[m] = rest[m].x;
    xw[m] = rest[m].x;
    rw[m] = D.r;
    r[m] = D.r;
    cb[m] = C.b;
    cx[m] = C.x;
    cdir[m] = C.dir;
    down[m] = GLevel{rest[m].h, rest[m].l - 1, C.b, C.x};
  }
  launches += group_sell(rest, 0, 0, b, nomask, x, rw, s);         // r = b - A x
  launches += group_sell(rest, 2, 3, b, cdir, r, cb, s);           // r_c = R r, coarse Dirichlet zeroed
  launches += group_vcycle(down, s);
  launches += group_sell(rest, 1, 2, x, nomask, cx, xw, s);        // x += P e_c
  launches += group_smooth(rest, false, s);
  return launches;
}

}  // namespace

struct vk_group {
  int max_members = 0;
  std::vector<GroupMember> m;
  int* dflags = nullptr;      // device: 2 flags per member
  int* hflags = nullptr;      // pinned host mirror
  int64_t launches = 0;
  ~vk_group() {
    if (dflags) cudaFree(dflags);
    if (hflags) cudaFreeHost(hflags);
  }
};

namespace {

// The tail of solve_impl for one member: x = Z y from the rotated Hessenberg system, true residual.
void group_finish(vk_group* g, GroupMember& M, cudaStream_t s) {
  vk_hierarchy* h = M.h;
  DevLevel& F = h->lv.back();
  const int n = F.ndof, ldh = h->kmax + 1, m = M.j;
  std::vector<double> Hh(size_t(ldh) * std::max(m, 1)), gh(m + 1), y(std::max(m, 1));
  M.hist.assign(m + 1, 0.0);
  CK(cudaMemcpyAsync(Hh.data(), h->H, size_t(ldh) * m * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(gh.data(), h->g, (m + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(M.hist.data(), h->hist, (m + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = m - 1; i >= 0; --i) {
    double acc = gh[i];
    for (int k = i + 1; k < m; ++k) acc -= Hh[size_t(k) * ldh + i] * y[k];
    y[i] = acc / Hh[size_t(i) * ldh + i];
  }
  CK(cudaMemcpyAsync(h->yv, y.data(), m * sizeof(double), cudaMemcpyHostToDevice, s));
  g->launches += vk::gpu::combine(h->Z, h->ldv, m, h->yv, M.x, n, s);
  g->launches += vk::gpu::copy(F.t, M.b, n, s);
  g->launches += vk::gpu::pressure_project(F.t, F.n_u, F.n_p, h->partial, h->scal + 1, s);
  g->launches += vk::gpu::sell_residual(F.A, F.t, M.x, F.r, s);
  g->launches += 2;
  M.true_res = std::sqrt(device_dot(h, F.r, F.r, n, s));
  if (M.status == VK_OK && !M.converged) M.status = VK_ERR_NOT_CONVERGED;
  M.active = false;
  h->in_group = false;
}

}  // namespace

extern "C" {

int vk_group_create(int max_members, vk_group** out) {
  return guard([&] {
    if (!out || max_members < 1 || max_members > vk::gpu::kGroupMax) raise(VK_ERR_ARG, "max_members must be in 1..24");
    *out = nullptr;
    auto g = std::make_unique<vk_group>();
    g->max_members = max_members;
    g->m.resize(max_members);
    std::lock_guard<std::mutex> lock(g_device_mu);
    CK(cudaMalloc(&g->dflags, 2 * sizeof(int) * max_members));
    CK(cudaMallocHost(&g->hflags, 2 * sizeof(int) * max_members));
    *out = g.release();
    return VK_OK;
  });
}

void vk_group_destroy(vk_group* g) {
  if (!g) return;
  std::lock_guard<std::mutex> lock(g_device_mu);
  cudaDeviceSynchronize();
  for (GroupMember& M : g->m)
    if (M.used && M.h) M.h->in_group = false;
  delete g;
}

int vk_group_launches(const vk_group* g, int64_t* launches) {
  return guard([&] {
    if (!g || !launches) raise(VK_ERR_ARG, "null argument");
    *launches = g->launches;
    return VK_OK;
  });
}

int vk_group_add(vk_group* g, vk_hierarchy* h, const double* b, double* x, double rtol, int maxit, void* stream,
                 int* member) {
  return guard([&] {
    if (!g || !member) raise(VK_ERR_ARG, "null argument");
    check_device(h);
    if (h->in_group) raise(VK_ERR_ARG, "hierarchy is already in a group member");
    if (!b || !x || b == x) raise(VK_ERR_ARG, "null or aliased vectors");
    if (maxit < 1 || maxit > h->kmax) raise(VK_ERR_ARG, "maxit must be in 1..max_iterations");
    if (!(rtol >= 0.0)) raise(VK_ERR_ARG, "rtol must be >= 0");
    for (const GroupMember& M : g->m)
      if (M.used && M.h && M.h->opt.factor_prec != h->opt.factor_prec)
        raise(VK_ERR_ARG, "group members must share factor_prec");
    int slot = -1;
    for (int i = 0; i < g->max_members; ++i)
      if (!g->m[i].used) {
        slot = i;
        break;
      }
    if (slot < 0) raise(VK_ERR_ARG, "group is full");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GroupMember M;
    M.h = h;
    M.b = b;
    M.x = x;
    M.rtol = rtol;
    M.maxit = maxit;
    M.used = true;
    M.t0 = std::chrono::steady_clock::now();
    // prologue of solve_impl: b_hat = projected b, beta, v_1 = b_hat / beta
    DevLevel& F = h->lv.back();
    const int n = F.ndof;
    g->launches += vk::gpu::copy(h->V, b, n, s);
    g->launches += vk::gpu::pressure_project(h->V, F.n_u, F.n_p, h->partial, h->scal + 1, s);
    g->launches += 2;
    M.beta = std::sqrt(device_dot(h, h->V, h->V, n, s));
    if (!std::isfinite(M.beta)) raise(VK_ERR_NONFINITE, "right-hand side is not finite");
    if (M.beta == 0.0) {
      g->launches += vk::gpu::fill(x, 0.0, n, s);
      CK(cudaStreamSynchronize(s));
      M.converged = true;
      M.hist.assign(1, 0.0);
      M.true_res = 0.0;
    } else {
      g->launches += vk::gpu::scale_copy(h->V, h->scal, h->V, n, s);
      g->launches += vk::gpu::fill(h->g, 0.0, h->kmax + 1, s);
      CK(cudaMemcpyAsync(h->g, &M.beta, sizeof(double), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(h->hist, &M.beta, sizeof(double), cudaMemcpyHostToDevice, s));
      CK(cudaGetLastError());
      M.active = true;
      h->in_group = true;
    }
    g->m[slot] = std::move(M);
    *member = slot;
    return VK_OK;
  });
}

int vk_group_step(vk_group* g, void* stream, int* active) {
  return guard([&] {
    if (!g) raise(VK_ERR_ARG, "null group");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int> act;
    for (int i = 0; i < g->max_members; ++i)
      if (g->m[i].used && g->m[i].active) act.push_back(i);
    if (!act.empty()) {
      const int cnt = int(act.size());
      std::vector<GLevel> fin(cnt);
      int kmax = 0;
      for (int c = 0; c < cnt; ++c) {
        GroupMember& M = g->m[act[c]];
        vk_hierarchy* h = M.h;
        fin[c] = GLevel{h, h->prob.nlevels - 1, h->V + h->ldv * M.j, h->Z + h->ldv * M.j};
        kmax = std::max(kmax, h->kmax);
        h->n_vcycle++;
      }
      g->launches += group_vcycle(fin, s);
      vk::gpu::GroupVecArgs pv, c1, c2, nw;
      pv.count = c1.count = c2.count = nw.count = cnt;
      std::vector<const double*> none(cnt, nullptr), zj(cnt);
      std::vector<const uint8_t*> nomask(cnt, nullptr);
      std::vector<double*> w(cnt);
      for (int c = 0; c < cnt; ++c) {
        GroupMember& M = g->m[act[c]];
        vk_hierarchy* h = M.h;
        DevLevel& F = h->lv.back();
        const int ldh = h->kmax + 1;
        double* z = h->Z + h->ldv * M.j;
        double* wv = h->V + h->ldv * (M.j + 1);
        double* hcol = h->H + int64_t(M.j) * ldh;
        zj[c] = z;
        w[c] = wv;
        pv.w[c] = z;
        pv.off[c] = F.n_u;
        pv.len[c] = F.n_p;
        pv.partial[c] = h->partial;
        pv.out[c] = h->scal + 1;
        for (vk::gpu::GroupVecArgs* a : {&c1, &c2, &nw}) {
          a->n[c] = F.ndof;
          a->V[c] = h->V;
          a->ld[c] = h->ldv;
          a->nvec[c] = M.j + 1;
          a->w[c] = wv;
          a->partial[c] = h->partial;
        }
        c1.out[c] = hcol;
        c2.out[c] = h->t2;
        c2.acc[c] = hcol;
        nw.out[c] = h->scal + 2;
      }
      g->launches += vk::gpu::group_pressure_project(pv, s);              // project z_j
      g->launches += group_sell(fin, 0, 1, none, nomask, zj, w, s);        // w = A z_j
      g->launches += vk::gpu::group_multi_dot(c1, s);                       // classical Gram-Schmidt, twice
      g->launches += vk::gpu::group_multi_axpy(c1, s);
      g->launches += vk::gpu::group_multi_dot(c2, s);
      g->launches += vk::gpu::group_multi_axpy(c2, s);
      g->launches += vk::gpu::group_norm2(nw, s);
      vk::gpu::GroupGivensArgs gv;
      gv.count = cnt;
      gv.kmax = kmax;
      for (int c = 0; c < cnt; ++c) {
        GroupMember& M = g->m[act[c]];
        vk_hierarchy* h = M.h;
        gv.H[c] = h->H;
        gv.ldh[c] = h->kmax + 1;
        gv.cs[c] = h->cs;
        gv.sn[c] = h->sn;
        gv.g[c] = h->g;
        gv.hist[c] = h->hist;
        gv.j[c] = M.j;
        gv.rtol[c] = M.rtol;
        gv.flag[c] = g->dflags + 2 * act[c];
        gv.wsq[c] = h->scal + 2;
        gv.w[c] = w[c];
        gv.vnext[c] = w[c];
        gv.n[c] = h->lv.back().ndof;
      }
      g->launches += vk::gpu::group_normalize_givens(gv, s);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(g->hflags, g->dflags, 2 * sizeof(int) * g->max_members, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int c = 0; c < cnt; ++c) {
        GroupMember& M = g->m[act[c]];
        M.j += 1;
        const int* f = g->hflags + 2 * act[c];
        if (f[1]) {
          M.status = VK_ERR_NONFINITE;
        } else if (f[0]) {
          M.converged = true;
        } else if (M.j < M.maxit) {
          continue;
        }
        group_finish(g, M, s);
      }
    }
    if (active) {
      int a = 0;
      for (const GroupMember& M : g->m) a += (M.used && M.active) ? 1 : 0;
      *active = a;
    }
    return VK_OK;
  });
}

int vk_group_add_host(vk_group* g, vk_hierarchy* h, const double* b_host, double rtol, int maxit, void* stream,
                      int* member) {
  return guard([&] {
    check_device(h);
    if (!b_host) raise(VK_ERR_ARG, "null right-hand side");
    if (h->in_group) raise(VK_ERR_ARG, "hierarchy is already in a group member");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = h->lv.back().ndof;
    CK(cudaMemcpyAsync(h->bh, b_host, size_t(n) * sizeof(double), cudaMemcpyHostToDevice, s));
    const int rc = vk_group_add(g, h, h->bh, h->xh, rtol, maxit, stream, member);
    if (rc != VK_OK) raise(rc, vk_last_error());
    return VK_OK;
  });
}

int vk_group_active(const vk_group* g, int member, int* active) {
  return guard([&] {
    if (!g || !active || member < 0 || member >= g->max_members || !g->m[member].used) raise(VK_ERR_ARG, "bad member");
    *active = g->m[member].active ? 1 : 0;
    return VK_OK;
  });
}

int vk_group_result(vk_group* g, int member, double* x_host, vk_solve_info* info) {
  return guard([&] {
    if (!g || member < 0 || member >= g->max_members) raise(VK_ERR_ARG, "bad member");
    GroupMember& M = g->m[member];
    if (!M.used || M.active) raise(VK_ERR_ARG, "member is not finished");
    if (x_host) {
      const int n = M.h->lv.back().ndof;
      CK(cudaMemcpy(x_host, M.x, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost));
    }
    if (info) {
      info->iterations = M.j;
      info->converged = M.converged ? 1 : 0;
      info->res0 = M.beta;
      info->res_est = M.hist.empty() ? 0.0 : M.hist.back();
      info->true_res = M.true_res;
      if (info->history)
        for (size_t i = 0; i < M.hist.size(); ++i) info->history[i] = M.hist[i];
      info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - M.t0).count();
    }
    const int st = M.status;
    if (st == VK_ERR_NONFINITE) g_err = "FGMRES residual estimate is not finite";
    if (st == VK_ERR_NOT_CONVERGED) g_err = "FGMRES did not reach rtol in maxit iterations";
    M = GroupMember{};
    return st;
  });
}

}  // extern "C"
