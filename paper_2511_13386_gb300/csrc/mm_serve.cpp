// Serving loop of the C ABI (serve_submit / serve_poll).
//
// Requests carry a full problem (parameters, parareal configuration, host
// initial data).  A scheduler thread admits queued requests while their
// device footprint fits the HBM budget and a slot is free, and runs each
// admitted solve with parareal_run on its own stream from a small pool of
// worker threads, so solves that arrive while others are on the GPU overlap
// on the device.  Results are copied to host memory owned by the server
// until polled.
#include <math.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "mm_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t ticket = 0;
  mm_params params{};
  mm_parareal_cfg cfg{};
  std::vector<double> rho0;
  std::vector<unsigned char> g0;
  size_t footprint = 0;
  Clock::time_point t_submit;
  // result
  bool done = false;
  mm_status status = MM_OK;
  std::vector<double> rho_T;
  int iterations = 0;
  int64_t latency_ns = 0;
  int64_t kinetic_updates = 0;
};

size_t footprint_of(const mm_params& p, const mm_parareal_cfg& c) {
  const size_t gsz = p.precision == MM_FP32G ? 4 : 8;
  const size_t N = c.n_slices;
  // slices (3 arrays of N+1 densities), fine inputs and double buffer,
  // fine column arrays, staging
  return 3 * (N + 1) * p.nx * 8 + 3 * N * (size_t)p.nx * p.nv * gsz + N * (size_t)p.nx * 512 +
         (size_t)p.nx * p.nv * gsz + (1u << 20);
}

}  // namespace

struct mm_server {
  mm_server_cfg cfg{};
  mm_alloc alloc{};
  bool has_alloc = false;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<std::shared_ptr<Job>> queue;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  size_t in_use = 0;
  int running = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread sched;
  std::vector<std::thread> workers;

  void run_job(std::shared_ptr<Job> j) {
    cudaSetDevice(device);
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    mm_ctx* ctx = nullptr;
    mm_status st = mm_create(&j->params, has_alloc ? &alloc : nullptr, &ctx);
    std::vector<double> slices((size_t)(j->cfg.n_slices + 1) * j->params.nx);
    mm_parareal_stats ps{};
    if (st == MM_OK) st = parareal_run(ctx, &j->cfg, j->rho0.data(), j->g0.data(), slices.data(), &ps, s);
    if (ctx) mm_destroy(ctx);
    cudaStreamDestroy(s);
    std::lock_guard<std::mutex> lk(mu);
    j->status = st;
    j->iterations = ps.iterations;
    j->kinetic_updates = ps.kinetic_updates;
    if (st == MM_OK)
      j->rho_T.assign(slices.end() - j->params.nx, slices.end());
    j->latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - j->t_submit).count();
    j->done = true;
    in_use -= j->footprint;
    --running;
    cv_done.notify_all();
    cv_sched.notify_all();
  }

  void scheduler() {
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      cv_sched.wait(lk, [&] {
        if (stop) return true;
        if (queue.empty()) return false;
        auto& j = queue.front();
        return running < cfg.max_slots && in_use + j->footprint <= cfg.hbm_budget_bytes;
      });
      if (stop) break;
      auto j = queue.front();
      queue.pop_front();
      in_use += j->footprint;
      ++running;
      // reap finished threads, then start this job
      workers.emplace_back([this, j] { run_job(j); });
    }
  }
};

extern "C" mm_status mm_server_create(const mm_server_cfg* cfg, const mm_alloc* alloc, mm_server** out) {
  if (!cfg || !out) return mm_fail(MM_ERR_INVALID, "NULL argument");
  if (cfg->max_slots < 1 || cfg->hbm_budget_bytes == 0)
    return mm_fail(MM_ERR_INVALID, "max_slots >= 1 and a non-zero budget are required");
  mm_server* s = new mm_server();
  s->cfg = *cfg;
  if (s->cfg.wait_limit_ms <= 0) s->cfg.wait_limit_ms = 60000;
  if (alloc && alloc->alloc && alloc->free) {
    s->alloc = *alloc;
    s->has_alloc = true;
  }
  cudaGetDevice(&s->device);
  s->sched = std::thread([s] { s->scheduler(); });
  *out = s;
  return MM_OK;
}

extern "C" mm_status serve_submit(mm_server* s, const mm_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return mm_fail(MM_ERR_INVALID, "NULL argument");
  if (!req->rho0 || !req->g0) return mm_fail(MM_ERR_INVALID, "request without initial data");
  const mm_params& p = req->params;
  if (p.nx < 8 || p.nv < 4 || req->cfg.n_slices < 1) return mm_fail(MM_ERR_INVALID, "bad request sizes");
  auto j = std::make_shared<Job>();
  j->params = p;
  j->cfg = req->cfg;
  j->rho0.assign(req->rho0, req->rho0 + p.nx);
  const size_t gb = (size_t)p.nx * p.nv * (p.precision == MM_FP32G ? 4 : 8);
  j->g0.resize(gb);
  memcpy(j->g0.data(), req->g0, gb);
  j->footprint = footprint_of(p, req->cfg);
  if (j->footprint > s->cfg.hbm_budget_bytes)
    return mm_fail(MM_ERR_INVALID, "request footprint exceeds the whole HBM budget");
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  j->ticket = s->next_ticket++;
  s->jobs[j->ticket] = j;
  s->queue.push_back(j);
  *ticket = j->ticket;
  s->cv_sched.notify_all();
  return MM_OK;
}

extern "C" mm_status serve_poll(mm_server* s, uint64_t ticket, mm_result* res, int32_t timeout_ms) {
  if (!s || !res) return mm_fail(MM_ERR_INVALID, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return mm_fail(MM_ERR_UNKNOWN_TICKET, "unknown ticket");
  auto j = it->second;
  if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, (int)timeout_ms)), [&] { return j->done; }))
    return mm_fail(MM_ERR_NOT_READY, "result not ready");
  res->status = j->status;
  res->iterations = j->iterations;
  res->latency_ns = j->latency_ns;
  res->kinetic_updates = j->kinetic_updates;
  if (res->rho_T && j->status == MM_OK) memcpy(res->rho_T, j->rho_T.data(), j->rho_T.size() * sizeof(double));
  s->jobs.erase(it);
  return MM_OK;
}

extern "C" mm_status mm_server_destroy(mm_server* s) {
  if (!s) return MM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& j : s->queue) {
      j->status = MM_ERR_INVALID;
      j->done = true;
    }
    s->queue.clear();
  }
  s->cv_sched.notify_all();
  if (s->sched.joinable()) s->sched.join();
  for (auto& t : s->workers)
    if (t.joinable()) t.join();
  s->cv_done.notify_all();
  delete s;
  return MM_OK;
}
