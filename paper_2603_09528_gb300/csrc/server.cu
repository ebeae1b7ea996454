// Request server with continuous batching on one device.  Declarations and
// contracts: include/tpt.h.
//
//   submit ──> setup queue ──(setup threads: plan through the eigenbasis
//              cache)──> ready set (by arrival) ──(slot threads: admit the
//              oldest ready request once it fits the memory budget)──> H2D,
//              solve, D2H on the slot's stream ──> done
//
// Every slot owns a CUDA stream, so the solves of admitted requests overlap on
// the device; a request that arrives while others run is admitted as soon as
// a slot and enough of the budget are free.  Request buffers are
// stream-ordered allocations from a memory pool of their own (plan tables
// come from another, so small tables never split the big blocks) and plans are
// created and destroyed without synchronising the device, so admitting or
// retiring one request never stalls the others.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <shared_mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cache.h"
#include "tpt_internal.h"

namespace {

struct Request {
  unsigned long long id = 0;
  tpt_desc desc{};
  std::vector<double> dxf[3], dxc[3];    // the descriptor's arrays, copied
  const double* f_host = nullptr;
  double* phi_host = nullptr;
  tpt_plan plan = nullptr;
  size_t npts = 0, work_bytes = 0, need = 0;
  tpt_result res{};
  bool done = false;
};

int cuda_st(cudaError_t e) {
  if (e == cudaSuccess) return TPT_OK;
  cudaGetLastError();
  tpt::note_cuda_error(e);
  return e == cudaErrorMemoryAllocation ? TPT_ERR_OOM : TPT_ERR_CUDA;
}

}  // namespace

struct tpt_server_s {
  tpt_server_config cfg{};
  tpt::BasisCache cache;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  std::mutex mu;
  std::mutex h2d_mu;   // one input copy at a time (see execute)
  // Solves of large requests (each fills the GPU) run one at a time, so that
  // the solve in progress has the device to itself while other slots copy;
  // smaller ones share the device
  std::shared_mutex compute_mu;
  static constexpr size_t kExclusivePoints = size_t(1) << 24;
  std::condition_variable cv_setup, cv_ready, cv_done;
  std::deque<Request*> setup_q;
  std::map<unsigned long long, Request*> ready;   // planned, ordered by arrival
  std::unordered_map<unsigned long long, std::unique_ptr<Request>> reqs;
  unsigned long long next_id = 1;
  size_t in_use = 0, peak = 0;
  int inflight = 0, peak_inflight = 0;
  unsigned long long submitted = 0, finished = 0, rejected = 0;
  bool stop = false;
  std::vector<std::thread> threads;

  explicit tpt_server_s(const tpt_server_config& c) : cfg(c), cache(c.cuda_device, c.cache_budget) {}

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  // caller holds mu
  void finish(Request* r, int status) {
    r->res.status = status;
    r->res.t_done = now();
    r->done = true;
    ++finished;
    if (status != TPT_OK && status != TPT_ERR_NOT_CONVERGED && r->res.t_admit == 0.0) ++rejected;
    cv_done.notify_all();
  }

  void setup_loop() {
    if (cfg.cuda_device >= 0) cudaSetDevice(cfg.cuda_device);
    for (;;) {
      Request* r = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_setup.wait(lk, [&] { return stop || !setup_q.empty(); });
        if (setup_q.empty()) return;   // stop with nothing left to plan
        r = setup_q.front();
        setup_q.pop_front();
      }
      tpt_plan p = nullptr;
      tpt::clear_cuda_error();
      int st = tpt::create_plan(&r->desc, cfg.cuda_device, &cache, &p);
      size_t wb = 0;
      if (st == TPT_OK) st = tpt_workspace_bytes(p, &wb);
      std::lock_guard<std::mutex> g(mu);
      r->res.t_planned = now();
      if (st != TPT_OK) {
        if (p) tpt_plan_destroy(p);
        r->res.failed_step = TPT_STEP_PLAN;
        r->res.cuda_error = static_cast<int>(tpt::last_cuda_error());
        finish(r, st);
        continue;
      }
      r->plan = p;
      r->work_bytes = wb;
      r->need = 2 * r->npts * sizeof(double) + wb + 3 * 256;
      r->res.device_bytes = r->need;
      if (r->need > cfg.memory_budget) {   // can never fit: reject rather than wait forever
        tpt_plan_destroy(p);
        r->plan = nullptr;
        finish(r, TPT_ERR_OOM);
        continue;
      }
      ready.emplace(r->id, r);
      cv_ready.notify_all();
    }
  }

  // H2D, solve, D2H on the slot's stream; returns the request's status and
  // records in r->res where a failure happened and its CUDA error.
  int execute(Request* r, cudaStream_t s) {
    tpt::clear_cuda_error();
    r->res.merged = 1;
    int step = 0;
    const int st = execute_steps(r, s, &step);
    if (st != TPT_OK && st != TPT_ERR_NOT_CONVERGED) {
      r->res.failed_step = step;
      r->res.cuda_error = static_cast<int>(tpt::last_cuda_error());
    }
    return st;
  }

  int execute_steps(Request* r, cudaStream_t s, int* step) {
    if (cfg.cuda_device < 0) {   // dry run: the solve is a sleep
      const double ns = cfg.dry_run_ns_per_point * static_cast<double>(r->npts);
      std::this_thread::sleep_for(std::chrono::nanoseconds(static_cast<long long>(ns)));
      return TPT_OK;
    }
    const size_t bytes = r->npts * sizeof(double);
    void* buf[3] = {nullptr, nullptr, nullptr};
    const size_t sz[3] = {bytes + 256, bytes + 256, r->work_bytes + 256};
    int st = TPT_OK;
    *step = TPT_STEP_ALLOC;
    for (int i = 0; i < 3 && st == TPT_OK; ++i)
      st = tpt::injected_alloc_failure() ? TPT_ERR_OOM
                                         : cuda_st(cudaMallocFromPoolAsync(&buf[i], sz[i], cache.buffer_pool(), s));
    auto aligned = [](void* p) {
      return reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 255) & ~static_cast<uintptr_t>(255));
    };
    if (st == TPT_OK) {
      double* f = reinterpret_cast<double*>(aligned(buf[0]));
      double* phi = reinterpret_cast<double*>(aligned(buf[1]));
      void* work = aligned(buf[2]);
      {
        // input copies take turns (in about admission order) instead of
        // sharing the host link, so that the oldest admitted request's solve
        // starts as early as possible and the next copy overlaps it
        std::lock_guard<std::mutex> g(h2d_mu);
        *step = TPT_STEP_H2D;
        st = cuda_st(cudaMemcpyAsync(f, r->f_host, bytes, cudaMemcpyHostToDevice, s));
        if (st == TPT_OK) st = cuda_st(cudaStreamSynchronize(s));
      }
      r->res.t_copied = now();
      if (st == TPT_OK) {
        *step = TPT_STEP_SOLVE;
        if (r->npts >= kExclusivePoints) {
          std::unique_lock<std::shared_mutex> g(compute_mu);
          st = tpt_solve(r->plan, f, phi, work, s, &r->res.info);
        } else {
          std::shared_lock<std::shared_mutex> g(compute_mu);
          st = tpt_solve(r->plan, f, phi, work, s, &r->res.info);
        }
        r->res.t_solved = now();
        if (st == TPT_OK || st == TPT_ERR_NOT_CONVERGED) {
          const int cs = cuda_st(cudaMemcpyAsync(r->phi_host, phi, bytes, cudaMemcpyDeviceToHost, s));
          if (cs != TPT_OK) {
            *step = TPT_STEP_D2H;
            st = cs;
          }
        }
      }
    }
    for (void* b : buf)
      if (b) cudaFreeAsync(b, s);
    const int ss = cuda_st(cudaStreamSynchronize(s));
    if (st == TPT_OK && ss != TPT_OK) *step = TPT_STEP_SYNC;
    return st != TPT_OK ? st : ss;
  }

  // Same-shape batching: requests that may join a group led by r.
  bool mergeable(const Request* r) const {
    if (cfg.merge <= 1 || r->npts >= kExclusivePoints || !r->plan) return false;
    const tpt_desc& d = r->desc;   // the grouped kernels' conditions (see tpt::group_eligible)
    if (d.precision != TPT_PREC_MIXED_BF16X3 || !(d.rtol > 0.0) || d.n[0] % 4 != 0 || d.n[2] > 512) return false;
    return cfg.cuda_device < 0 || tpt::group_eligible(r->plan);
  }
  static bool same_shape(const Request* a, const Request* b) {
    return a->desc.n[0] == b->desc.n[0] && a->desc.n[1] == b->desc.n[1] && a->desc.n[2] == b->desc.n[2] &&
           a->desc.precision == b->desc.precision;
  }
  static constexpr size_t kGroupExtra = 16384;   // per request: job tables and scalars of a group
  static constexpr size_t kMinGroup = 3;          // smallest group worth solving together

  // The requests of `grp` solved together as one grouped batch on stream s;
  // fills each request's result times and info, returns their statuses.
  std::vector<int> execute_group(const std::vector<Request*>& grp, cudaStream_t s) {
    const int n = static_cast<int>(grp.size());
    std::vector<int> st(n, TPT_OK);
    for (Request* r : grp) r->res.merged = n;
    if (cfg.cuda_device < 0) {   // dry run: one sleep for all their points
      double pts = 0.0;
      for (Request* r : grp) pts += static_cast<double>(r->npts);
      std::this_thread::sleep_for(std::chrono::nanoseconds(static_cast<long long>(cfg.dry_run_ns_per_point * pts)));
      return st;
    }
    std::vector<tpt_plan_s*> plans;
    for (Request* r : grp) plans.push_back(r->plan);
    tpt::GroupSolve* g = tpt::group_create(plans.data(), n);
    if (!g) {   // cannot be grouped after all: one after another
      for (int i = 0; i < n; ++i) st[i] = execute(grp[i], s);
      return st;   // (execute records each as solved alone)
    }
    tpt::clear_cuda_error();
    int step = TPT_STEP_ALLOC;
    std::vector<void*> bufs;
    auto alloc = [&](size_t bytes, void** out) -> int {
      if (tpt::injected_alloc_failure()) return TPT_ERR_OOM;
      const int e = cuda_st(cudaMallocFromPoolAsync(out, bytes + 256, cache.buffer_pool(), s));
      if (e == TPT_OK) bufs.push_back(*out);
      return e;
    };
    auto aligned = [](void* p) {
      return reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 255) & ~static_cast<uintptr_t>(255));
    };
    std::vector<const double*> fs(n);
    std::vector<double*> phis(n);
    void* work = nullptr;
    void* tables = nullptr;
    void* scal = nullptr;
    int gs = TPT_OK;
    for (int i = 0; i < n && gs == TPT_OK; ++i) {
      void* a = nullptr;
      void* b = nullptr;
      gs = alloc(grp[i]->npts * sizeof(double), &a);
      if (gs == TPT_OK) gs = alloc(grp[i]->npts * sizeof(double), &b);
      if (gs == TPT_OK) {
        fs[i] = reinterpret_cast<const double*>(aligned(a));
        phis[i] = reinterpret_cast<double*>(aligned(b));
      }
    }
    if (gs == TPT_OK) gs = alloc(tpt::group_workspace_bytes(g), &work);
    if (gs == TPT_OK) gs = alloc(tpt::group_table_bytes(g), &tables);
    if (gs == TPT_OK) gs = alloc(static_cast<size_t>(n) * 16 * sizeof(double), &scal);
    if (gs == TPT_OK) {
      std::lock_guard<std::mutex> lk(h2d_mu);   // input copies take turns (see execute)
      step = TPT_STEP_H2D;
      for (int i = 0; i < n && gs == TPT_OK; ++i)
        gs = cuda_st(cudaMemcpyAsync(const_cast<double*>(fs[i]), grp[i]->f_host, grp[i]->npts * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
      if (gs == TPT_OK) gs = cuda_st(cudaStreamSynchronize(s));
    }
    const double tc = now();
    for (Request* r : grp) r->res.t_copied = tc;
    std::vector<double> h(static_cast<size_t>(n) * 16, 0.0);
    if (gs == TPT_OK) {
      std::shared_lock<std::shared_mutex> lk(compute_mu);
      step = TPT_STEP_SOLVE;
      tpt::group_set_memory(g, aligned(tables), tpt::group_table_bytes(g));
      gs = tpt::group_prepare(g, fs.data(), phis.data(), aligned(work), s);
      if (gs == TPT_OK) gs = tpt::group_solve_adaptive(g, reinterpret_cast<double*>(aligned(scal)), h.data(), s);
    }
    const double ts = now();
    for (int i = 0; i < n; ++i) {
      Request* r = grp[i];
      if (gs != TPT_OK) {
        st[i] = gs;
        continue;
      }
      r->res.t_solved = ts;
      st[i] = tpt::solve_info(r->plan, h.data() + 16 * i, &r->res.info);
      if (st[i] == TPT_OK || st[i] == TPT_ERR_NOT_CONVERGED) {
        const int cs = cuda_st(cudaMemcpyAsync(r->phi_host, phis[i], r->npts * sizeof(double),
                                               cudaMemcpyDeviceToHost, s));
        if (cs != TPT_OK) {
          st[i] = cs;
          r->res.failed_step = TPT_STEP_D2H;
          r->res.cuda_error = static_cast<int>(tpt::last_cuda_error());
        }
      }
    }
    for (void* b : bufs) cudaFreeAsync(b, s);
    const int ss = cuda_st(cudaStreamSynchronize(s));
    tpt::group_destroy(g);
    for (int i = 0; i < n; ++i) {
      if (st[i] == TPT_OK && ss != TPT_OK) {
        st[i] = ss;
        grp[i]->res.failed_step = TPT_STEP_SYNC;
      }
      if (gs != TPT_OK) {
        grp[i]->res.failed_step = step;
        grp[i]->res.cuda_error = static_cast<int>(tpt::last_cuda_error());
      }
    }
    return st;
  }

  void slot_loop() {
    cudaStream_t s = nullptr;
    if (cfg.cuda_device >= 0) {
      cudaSetDevice(cfg.cuda_device);
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) cudaGetLastError();
    }
    for (;;) {
      std::vector<Request*> grp;
      size_t charged = 0;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_ready.wait(lk, [&] {
          if (!ready.empty() && in_use + ready.begin()->second->need <= cfg.memory_budget) return true;
          return stop && ready.empty() && setup_q.empty();
        });
        if (ready.empty()) break;
        Request* r = ready.begin()->second;   // the oldest planned request
        ready.erase(ready.begin());
        grp.push_back(r);
        charged = r->need;
        if (mergeable(r)) {   // other ready requests of its shape join it
          for (auto it = ready.begin(); it != ready.end() && static_cast<int>(grp.size()) < cfg.merge;) {
            Request* q = it->second;
            const size_t add = q->need + kGroupExtra;
            if (same_shape(q, r) && mergeable(q) && in_use + charged + add + kGroupExtra <= cfg.memory_budget) {
              grp.push_back(q);
              charged += add;
              it = ready.erase(it);
            } else {
              ++it;
            }
          }
          // a pair gains less than the grouped path's set-up costs (measured:
          // groups of two served slower than the requests alone on four slots)
          if (grp.size() > 1 && grp.size() < kMinGroup) {
            for (size_t k = 1; k < grp.size(); ++k) ready.emplace(grp[k]->id, grp[k]);
            grp.resize(1);
            charged = r->need;
          }
          if (grp.size() > 1) charged += kGroupExtra;
        }
        in_use += charged;
        peak = in_use > peak ? in_use : peak;
        inflight += static_cast<int>(grp.size());
        peak_inflight = inflight > peak_inflight ? inflight : peak_inflight;
        const double ta = now();
        for (Request* q : grp) q->res.t_admit = ta;
      }
      std::vector<int> st;
      if (cfg.cuda_device >= 0 && !s) st.assign(grp.size(), TPT_ERR_CUDA);
      else if (grp.size() == 1) st.push_back(execute(grp[0], s));
      else st = execute_group(grp, s);
      for (Request* q : grp) {
        tpt_plan p = q->plan;
        q->plan = nullptr;
        if (p) tpt_plan_destroy(p);   // stream-ordered frees: no device synchronisation
      }
      cache.trim();
      {
        std::lock_guard<std::mutex> g(mu);
        in_use -= charged;
        inflight -= static_cast<int>(grp.size());
        for (size_t i = 0; i < grp.size(); ++i) finish(grp[i], st[i]);
        cv_ready.notify_all();      // freed memory may admit the next request
      }
    }
    if (s) cudaStreamDestroy(s);
  }
};

extern "C" {

int tpt_server_create(const tpt_server_config* cfg, tpt_server* out) {
  if (!out) return TPT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg || cfg->slots < 1 || cfg->setup_threads < 1 || cfg->memory_budget == 0 || cfg->slots > 64 ||
      cfg->setup_threads > 64 || !(cfg->dry_run_ns_per_point >= 0.0) || cfg->merge < 0 || cfg->merge > 256)
    return TPT_ERR_INVALID_ARG;
  if (cfg->cuda_device >= 0) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
      cudaGetLastError();
      return TPT_ERR_CUDA;
    }
    if (cfg->cuda_device >= ndev) return TPT_ERR_INVALID_ARG;
    cudaSetDevice(cfg->cuda_device);
  }
  tpt_server s = new (std::nothrow) tpt_server_s(*cfg);
  if (!s) return TPT_ERR_OOM;
  const int st = s->cache.init();
  if (st != TPT_OK) {
    delete s;
    return st;
  }
  for (int i = 0; i < cfg->setup_threads; ++i) s->threads.emplace_back([s] { s->setup_loop(); });
  for (int i = 0; i < cfg->slots; ++i) s->threads.emplace_back([s] { s->slot_loop(); });
  *out = s;
  return TPT_OK;
}

int tpt_server_submit(tpt_server s, const tpt_desc* desc, const double* f_host, double* phi_host,
                      unsigned long long* ticket) {
  if (!s || !desc || !f_host || !phi_host || !ticket) return TPT_ERR_INVALID_ARG;
  auto r = std::unique_ptr<Request>(new (std::nothrow) Request);
  if (!r) return TPT_ERR_OOM;
  r->desc = *desc;
  size_t npts = 1;
  for (int d = 0; d < 3; ++d) {
    if (desc->n[d] < 1 || !desc->dxf[d] || !desc->dxc[d]) return TPT_ERR_INVALID_ARG;
    r->dxf[d].assign(desc->dxf[d], desc->dxf[d] + desc->n[d]);
    r->dxc[d].assign(desc->dxc[d], desc->dxc[d] + desc->n[d] + 1);
    r->desc.dxf[d] = r->dxf[d].data();
    r->desc.dxc[d] = r->dxc[d].data();
    npts *= static_cast<size_t>(desc->n[d]);
  }
  r->npts = npts;
  r->f_host = f_host;
  r->phi_host = phi_host;
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stop) return TPT_ERR_INVALID_ARG;
  r->id = s->next_id++;
  r->res.t_submit = s->now();
  *ticket = r->id;
  s->setup_q.push_back(r.get());
  s->reqs.emplace(r->id, std::move(r));
  ++s->submitted;
  s->cv_setup.notify_one();
  return TPT_OK;
}

int tpt_server_warm(tpt_server s, const tpt_desc* desc) {
  if (!s || !desc) return TPT_ERR_INVALID_ARG;
  if (s->cfg.cuda_device >= 0) cudaSetDevice(s->cfg.cuda_device);
  tpt_plan p = nullptr;
  int st = tpt::create_plan(desc, s->cfg.cuda_device, &s->cache, &p);
  size_t wb = 0;
  if (st == TPT_OK && p && s->cfg.cuda_device >= 0) st = tpt_workspace_bytes(p, &wb);
  if (p) tpt_plan_destroy(p);   // the plan was never used: its tables can go at once
  if (st != TPT_OK || s->cfg.cuda_device < 0) return st;
  // grow the memory pool to hold `slots` requests of this shape (the
  // buffers execute() takes), so that the first requests do not wait for the
  // driver to map memory; the pool keeps what is freed
  const size_t npts = static_cast<size_t>(desc->n[0]) * desc->n[1] * desc->n[2];
  const size_t sz[3] = {npts * sizeof(double) + 256, npts * sizeof(double) + 256, wb + 256};
  const size_t need = sz[0] + sz[1] + sz[2];
  const int sets = static_cast<int>(std::min<size_t>(static_cast<size_t>(s->cfg.slots), s->cfg.memory_budget / need));
  cudaStream_t ws = nullptr;
  if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return TPT_OK;   // only a warm-up: requests will grow the pool themselves
  }
  std::vector<void*> bufs;
  for (int k = 0; k < sets; ++k)
    for (size_t b : sz) {
      void* ptr = nullptr;
      if (cudaMallocFromPoolAsync(&ptr, b, s->cache.buffer_pool(), ws) != cudaSuccess) {
        cudaGetLastError();
        break;
      }
      bufs.push_back(ptr);
    }
  for (void* b : bufs) cudaFreeAsync(b, ws);
  cudaStreamSynchronize(ws);
  cudaStreamDestroy(ws);
  cudaGetLastError();
  return TPT_OK;
}

int tpt_server_wait(tpt_server s, unsigned long long ticket, double timeout_s, tpt_result* result) {
  if (!s || !result) return TPT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return TPT_ERR_INVALID_ARG;
  Request* r = it->second.get();
  auto pred = [&] { return r->done; };
  if (timeout_s < 0.0) {
    s->cv_done.wait(lk, pred);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
    return TPT_PENDING;
  }
  *result = r->res;
  s->reqs.erase(it);
  return TPT_OK;
}

int tpt_server_now(tpt_server s, double* t) {
  if (!s || !t) return TPT_ERR_INVALID_ARG;
  *t = s->now();
  return TPT_OK;
}

int tpt_server_stats(tpt_server s, tpt_serving_stats* out) {
  if (!s || !out) return TPT_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  s->cache.stats(&out->cache_hits, &out->cache_misses, &out->cache_bytes, nullptr);
  std::lock_guard<std::mutex> g(s->mu);
  out->submitted = s->submitted;
  out->completed = s->finished;
  out->rejected = s->rejected;
  out->peak_bytes = s->peak;
  out->peak_inflight = s->peak_inflight;
  return TPT_OK;
}

int tpt_server_destroy(tpt_server s) {
  if (!s) return TPT_ERR_INVALID_ARG;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->finished == s->submitted; });
    s->stop = true;
  }
  s->cv_setup.notify_all();
  s->cv_ready.notify_all();
  for (std::thread& t : s->threads) t.join();
  if (s->cfg.cuda_device >= 0) cudaSetDevice(s->cfg.cuda_device);
  delete s;
  return TPT_OK;
}

}  // extern "C"
