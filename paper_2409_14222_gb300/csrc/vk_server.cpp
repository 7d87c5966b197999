// Solve service on one GPU (include/vk.h, vk_server_*): a FIFO of Stokes solve requests of mixed mesh
// size and order.  `slots` worker threads find or build each request's hierarchy; then either group
// engines advance the admitted requests together as members of group solves (VK_SERVE_GROUP: one
// engine per size bucket, each with its own stream; one launch per stage of every FGMRES iteration over
// the bucket's members, requests joining and leaving between iterations), or each worker solves its
// request alone on its own CUDA stream (VK_SERVE_STREAMS).  Hierarchies are kept resident between requests
// in a pool keyed by the whole problem (N_coarse, nlevels, k and the bits of the viscosity nu, which
// enters the matrix); a pool entry is used by one slot at a time.  Admission is
// by device footprint (vk_footprint): when the budget would be exceeded, idle hierarchies are evicted
// least-recently-used first; a request waits while the memory it needs is held by busy solves.
//
// Built only on the public C ABI (vk_setup / vk_solve_host / vk_group_* / vk_footprint / vk_destroy):
// every request runs the same deterministic arithmetic on its own hierarchy, so a result does not
// depend on what else is being served.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "vk.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0, Clock::time_point t1) {
  return std::chrono::duration<double, std::milli>(t1 - t0).count();
}

// N_coarse, nlevels, k, cell type, bit pattern of nu (two requests share a hierarchy only if their
// matrices are the same; bc and domain have a single accepted value each, checked at submission)
using Key = std::tuple<int, int, int, int, uint64_t>;

Key key_of(const vk_problem& p) {
  uint64_t bits = 0;
  static_assert(sizeof(bits) == sizeof(p.nu), "nu is a double");
  std::memcpy(&bits, &p.nu, sizeof(bits));
  return Key{p.N_coarse, p.nlevels, p.k, p.cell, bits};
}

struct Instance {
  vk_hierarchy* h = nullptr;
  size_t bytes = 0;
  bool busy = false;
  Clock::time_point last_used;
};

struct Job {
  uint64_t ticket = 0;
  vk_problem problem{};
  std::vector<double> b;
  double rtol = 1e-8;
  int maxit = 100;
  Clock::time_point submitted;
};

struct Done {
  vk_result res{};
  std::vector<double> x;
};

}  // namespace

// Size buckets of the group engines (finest-level DoFs): below 2^16, below 2^19, larger.
constexpr int kBuckets = 3;
int bucket_of(size_t ndof) { return ndof < (size_t(1) << 16) ? 0 : ndof < (size_t(1) << 19) ? 1 : 2; }

// A request whose hierarchy is ready, waiting to join a group solve (VK_SERVE_GROUP).
struct Ready {
  Job job;
  Instance* inst = nullptr;
  double setup_ms = 0.0;
  Clock::time_point t_start;
};

struct vk_server {
  vk_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work;   // workers: new job or freed memory
  std::condition_variable cv_done;   // waiters: a result arrived
  std::condition_variable cv_engine; // group engines: a request became ready, or stop
  // VK_SERVE_GROUP: requests with a hierarchy, not yet members, one queue per size bucket; each bucket
  // has its own engine (group solve and stream), so requests of similar size share launches while
  // small requests do not advance at the pace of large ones
  std::deque<Ready> ready[kBuckets];
  int inflight = 0;                  // VK_SERVE_GROUP: requests taken by workers and not finished
  std::vector<std::thread> engines;
  std::deque<Job> queue;
  std::map<Key, std::vector<std::unique_ptr<Instance>>> pool;
  std::map<uint64_t, Done> done;
  std::vector<std::thread> workers;
  uint64_t next_ticket = 1;
  size_t used = 0;
  bool stopping = false;
  vk_server_stats st{};
  std::string error;
};

namespace {

thread_local std::string g_srv_err;

size_t footprint_of(vk_server* s, const vk_problem& p) {
  size_t b = 0;
  if (vk_footprint(&p, &s->cfg.options, &b) != VK_OK) return 0;
  return b;
}

// Called with s->mu held.  Returns an idle instance for key (marked busy), builds one if memory
// allows (evicting idle LRU instances), or returns nullptr if the request must wait.
Instance* acquire(vk_server* s, std::unique_lock<std::mutex>& lk, const vk_problem& p, int stream_id,
                  cudaStream_t stream, double* setup_ms, int* status) {
  const Key key = key_of(p);
  auto& list = s->pool[key];
  for (auto& inst : list)
    if (!inst->busy) {
      inst->busy = true;
      return inst.get();
    }
  // all instances of this key are busy: wait for one rather than build beyond the per-key cap
  if (int(list.size()) >= s->cfg.max_per_key) return nullptr;
  const size_t need = footprint_of(s, p);
  if (need == 0) {
    *status = VK_ERR_ARG;
    return nullptr;
  }
  if (need > s->cfg.memory_budget) {
    *status = VK_ERR_NO_MEMORY;
    return nullptr;
  }
  while (s->used + need > s->cfg.memory_budget) {
    // evict the least recently used idle instance of any key
    Instance* victim = nullptr;
    Key vkey{};
    for (auto& kv : s->pool)
      for (auto& inst : kv.second)
        if (!inst->busy && (!victim || inst->last_used < victim->last_used)) {
          victim = inst.get();
          vkey = kv.first;
        }
    if (!victim) return nullptr;  // everything resident is busy: wait for a release
    auto& vl = s->pool[vkey];
    for (size_t i = 0; i < vl.size(); ++i)
      if (vl[i].get() == victim) {
        vk_hierarchy* h = victim->h;
        s->used -= victim->bytes;
        vl.erase(vl.begin() + long(i));
        lk.unlock();
        vk_destroy(h);
        lk.lock();
        s->st.evictions++;
        break;
      }
  }
  // reserve the memory, build outside the lock
  s->used += need;
  auto inst = std::make_unique<Instance>();
  inst->busy = true;
  inst->bytes = need;
  Instance* raw = inst.get();
  s->pool[key].push_back(std::move(inst));
  lk.unlock();
  const auto t0 = Clock::now();
  vk_hierarchy* h = nullptr;
  const int rc = vk_setup(&p, &s->cfg.options, nullptr, stream, &h);
  *setup_ms = ms_since(t0, Clock::now());
  lk.lock();
  (void)stream_id;
  if (rc != VK_OK) {
    auto& l2 = s->pool[key];
    for (size_t i = 0; i < l2.size(); ++i)
      if (l2[i].get() == raw) {
        l2.erase(l2.begin() + long(i));
        break;
      }
    s->used -= need;
    *status = rc;
    // the released reservation may be what another worker is waiting for
    s->cv_work.notify_all();
    return nullptr;
  }
  raw->h = h;
  s->st.builds++;
  return raw;
}

// Records a finished request (called with s->mu held).
void complete(vk_server* s, uint64_t ticket, Done&& out) {
  s->st.completed++;
  if (out.res.status != VK_OK && out.res.status != VK_ERR_NOT_CONVERGED) s->st.failed++;
  s->done[ticket] = std::move(out);
  s->cv_done.notify_all();
}

// Builder / solver threads.  Each takes the next request, finds or builds its hierarchy (acquire),
// then either solves it alone on its own stream (VK_SERVE_STREAMS) or hands it to the group engine
// (VK_SERVE_GROUP, at most `slots` requests in flight).
void worker(vk_server* s, int id) {
  cudaSetDevice(s->cfg.device);
  cudaStream_t stream = nullptr;
  const bool stream_ok = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess;
  const bool group = s->cfg.mode == VK_SERVE_GROUP;
  // host staging is pageable: pinned allocations or frees at run time would synchronise the device
  std::vector<double> hx;
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv_work.wait(lk, [&] {
      return s->stopping || (!s->queue.empty() && (!group || s->inflight < s->cfg.slots));
    });
    if (s->stopping && s->queue.empty()) break;
    if (s->queue.empty() || (group && s->inflight >= s->cfg.slots)) continue;
    Job job = std::move(s->queue.front());
    s->queue.pop_front();
    if (group) s->inflight++;
    const auto t_start = Clock::now();
    double setup_ms = 0.0;
    int status = VK_OK;
    Instance* inst = nullptr;
    if (!stream_ok) status = VK_ERR_CUDA;
    while (status == VK_OK) {
      inst = acquire(s, lk, job.problem, id, stream, &setup_ms, &status);
      if (inst || status != VK_OK) break;
      if (s->stopping) {
        status = VK_ERR_CANCELLED;  // the service stopped while this request waited for memory
        break;
      }
      s->cv_work.wait(lk);  // memory held by busy solves: wait for a release
    }
    if (inst && group) {
      Ready r;
      r.job = std::move(job);
      r.inst = inst;
      r.setup_ms = setup_ms;
      r.t_start = t_start;
      const int bk = bucket_of(r.job.b.size());
      s->ready[bk].push_back(std::move(r));
      s->cv_engine.notify_all();
      continue;
    }
    Done out;
    out.res.queue_ms = ms_since(job.submitted, t_start);
    out.res.setup_ms = setup_ms;
    if (inst) {
      lk.unlock();
      const size_t n = job.b.size();
      hx.assign(n, 0.0);
      vk_solve_info info{};
      status = vk_solve_host(inst->h, job.b.data(), hx.data(), job.rtol, job.maxit, &info, stream);
      out.x = hx;
      out.res.iterations = info.iterations;
      out.res.converged = info.converged;
      out.res.res0 = info.res0;
      out.res.true_res = info.true_res;
      out.res.solve_ms = info.solve_ms;
      lk.lock();
      inst->busy = false;
      inst->last_used = Clock::now();
      s->cv_work.notify_all();
    }
    out.res.status = status;
    out.res.latency_ms = ms_since(job.submitted, Clock::now());
    if (group) {
      s->inflight--;
      s->cv_work.notify_all();
      s->cv_engine.notify_all();
    }
    complete(s, job.ticket, std::move(out));
  }
  lk.unlock();
  if (stream_ok) cudaStreamDestroy(stream);
}

// VK_SERVE_GROUP engine: admits ready requests as members of one group solve between iterations,
// advances all members by one FGMRES iteration per step (one launch per stage), and retires the
// members that finish.
void engine(vk_server* s, int bk) {
  cudaSetDevice(s->cfg.device);
  cudaStream_t stream = nullptr;
  const bool stream_ok = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess;
  const int maxm = std::min(s->cfg.slots, 24);
  vk_group* g = nullptr;
  const bool group_ok = stream_ok && vk_group_create(maxm, &g) == VK_OK;
  struct Active {
    Job job;
    Instance* inst;
    double setup_ms, queue_ms;
    Clock::time_point t_admit;
  };
  std::map<int, Active> act;
  auto finish = [&](Active& a, int status, Done&& out) {
    out.res.status = status;
    out.res.setup_ms = a.setup_ms;
    out.res.queue_ms = a.queue_ms;
    out.res.solve_ms = ms_since(a.t_admit, Clock::now());
    out.res.latency_ms = ms_since(a.job.submitted, Clock::now());
    std::lock_guard<std::mutex> lk(s->mu);
    a.inst->busy = false;
    a.inst->last_used = Clock::now();
    s->inflight--;
    s->cv_work.notify_all();
    complete(s, a.job.ticket, std::move(out));
  };
  while (true) {
    std::vector<Ready> adm;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto& rq = s->ready[bk];
      s->cv_engine.wait(lk, [&] {
        return !act.empty() || !rq.empty() || (s->stopping && s->inflight == 0 && s->queue.empty());
      });
      if (act.empty() && rq.empty() && s->stopping && s->inflight == 0 && s->queue.empty()) break;
      while (!rq.empty() && int(act.size() + adm.size()) < maxm) {
        adm.push_back(std::move(rq.front()));
        rq.pop_front();
      }
    }
    for (Ready& r : adm) {
      Active a{std::move(r.job), r.inst, r.setup_ms, 0.0, Clock::now()};
      a.queue_ms = ms_since(a.job.submitted, a.t_admit);   // submission -> joining the group
      int mid = -1;
      const int rc = group_ok ? vk_group_add_host(g, a.inst->h, a.job.b.data(), a.job.rtol, a.job.maxit, stream, &mid)
                              : VK_ERR_CUDA;
      if (rc != VK_OK) {
        finish(a, rc, Done{});
        continue;
      }
      act.emplace(mid, std::move(a));
    }
    if (act.empty()) continue;
    int nact = 0;
    const int rc = vk_group_step(g, stream, &nact);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->st.group_steps++;
      s->st.member_steps += int64_t(act.size());
    }
    std::vector<int> gone;
    for (auto& kv : act) {
      int still = 1;
      if (rc == VK_OK && vk_group_active(g, kv.first, &still) == VK_OK && still) continue;
      Done out;
      vk_solve_info info{};
      int st = rc;
      if (rc == VK_OK) {
        out.x.assign(kv.second.job.b.size(), 0.0);
        st = vk_group_result(g, kv.first, out.x.data(), &info);
        out.res.iterations = info.iterations;
        out.res.converged = info.converged;
        out.res.res0 = info.res0;
        out.res.true_res = info.true_res;
      }
      finish(kv.second, st, std::move(out));
      gone.push_back(kv.first);
    }
    for (int m : gone) act.erase(m);
    if (rc != VK_OK && group_ok) {
      // a failed step leaves the group's members in an unknown state: start a fresh group
      vk_group_destroy(g);
      g = nullptr;
      if (vk_group_create(maxm, &g) != VK_OK) g = nullptr;
    }
  }
  if (g) vk_group_destroy(g);
  if (stream_ok) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

void vk_default_server_config(vk_server_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->slots = 4;
  c->max_per_key = 2;
  c->memory_budget = 0;
  c->device = 0;
  c->mode = VK_SERVE_GROUP;
  vk_default_options(&c->options);
}

int vk_server_create(const vk_server_config* cfg, vk_server** out) {
  g_srv_err.clear();
  if (!cfg || !out || cfg->slots < 1 || cfg->slots > 64 || (cfg->mode != VK_SERVE_GROUP && cfg->mode != VK_SERVE_STREAMS) ||
      (cfg->mode == VK_SERVE_GROUP && cfg->slots > 24)) {
    g_srv_err = "bad server configuration";
    return VK_ERR_ARG;
  }
  auto s = std::make_unique<vk_server>();
  s->cfg = *cfg;
  if (s->cfg.max_per_key < 1) s->cfg.max_per_key = s->cfg.slots;
  s->cfg.options.lambdas = nullptr;
  s->cfg.options.host_only = 0;
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    cudaGetLastError();
    g_srv_err = "cudaSetDevice failed";
    return VK_ERR_CUDA;
  }
  if (s->cfg.memory_budget == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      g_srv_err = "cudaMemGetInfo failed";
      return VK_ERR_CUDA;
    }
    s->cfg.memory_budget = free_b / 10 * 6;
  }
  vk_server* raw = s.get();
  for (int i = 0; i < cfg->slots; ++i) raw->workers.emplace_back(worker, raw, i);
  if (raw->cfg.mode == VK_SERVE_GROUP)
    for (int bk = 0; bk < kBuckets; ++bk) raw->engines.emplace_back(engine, raw, bk);
  *out = s.release();
  return VK_OK;
}

int vk_server_submit(vk_server* s, const vk_request* r, uint64_t* ticket) {
  g_srv_err.clear();
  if (!s || !r || !r->b || !ticket || r->maxit < 1 || r->maxit > s->cfg.options.max_iterations ||
      !(r->rtol >= 0.0)) {
    g_srv_err = "bad request";
    return VK_ERR_ARG;
  }
  // the same checks as vk_setup (level count, index range of the finest mesh, viscosity, bc, domain)
  // before the size of b is computed from the problem
  if (vk_check_problem(&r->problem, &s->cfg.options) != VK_OK) {
    g_srv_err = std::string("bad problem: ") + vk_last_error();
    return VK_ERR_ARG;
  }
  const int k = r->problem.k;
  const int64_t Nf = int64_t(r->problem.N_coarse) << (r->problem.nlevels - 1);
  const int64_t ndof = 2 * (k * Nf + 1) * (k * Nf + 1) + ((k - 1) * Nf + 1) * ((k - 1) * Nf + 1);
  Job job;
  job.problem = r->problem;
  job.b.assign(r->b, r->b + ndof);
  job.rtol = r->rtol;
  job.maxit = r->maxit;
  job.submitted = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  job.ticket = s->next_ticket++;
  *ticket = job.ticket;
  s->queue.push_back(std::move(job));
  s->st.submitted++;
  s->cv_work.notify_one();
  return VK_OK;
}

int vk_server_wait(vk_server* s, uint64_t ticket, double* x_host, vk_result* res, int timeout_ms) {
  g_srv_err.clear();
  if (!s) return VK_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] { return s->done.count(ticket) > 0; };
  if (timeout_ms < 0)
    s->cv_done.wait(lk, ready);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return VK_ERR_TIMEOUT;
  Done d = std::move(s->done[ticket]);
  s->done.erase(ticket);
  lk.unlock();
  if (x_host && !d.x.empty()) std::memcpy(x_host, d.x.data(), d.x.size() * sizeof(double));
  if (res) *res = d.res;
  return VK_OK;
}

int vk_server_cancel(vk_server* s, uint64_t ticket) {
  g_srv_err.clear();
  if (!s) return VK_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
    if (it->ticket == ticket) {
      Done d;
      d.res.status = VK_ERR_CANCELLED;
      d.res.queue_ms = d.res.latency_ms = ms_since(it->submitted, Clock::now());
      s->queue.erase(it);
      s->st.completed++;
      s->st.failed++;
      s->done[ticket] = std::move(d);
      s->cv_done.notify_all();
      return VK_OK;
    }
  g_srv_err = "ticket is not queued (unknown, running or finished)";
  return VK_ERR_ARG;
}

int vk_server_get_stats(vk_server* s, vk_server_stats* out) {
  if (!s || !out) return VK_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->resident = 0;
  for (auto& kv : s->pool) out->resident += int32_t(kv.second.size());
  out->bytes_used = s->used;
  out->memory_budget = s->cfg.memory_budget;
  out->queued = int32_t(s->queue.size());
  return VK_OK;
}

void vk_server_destroy(vk_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->cv_engine.notify_all();
  }
  for (auto& t : s->engines) t.join();
  for (auto& kv : s->pool)
    for (auto& inst : kv.second)
      if (inst->h) vk_destroy(inst->h);
  delete s;
}

}  // extern "C"
