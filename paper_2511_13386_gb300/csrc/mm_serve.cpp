// Serving loop of the C ABI (serve_submit / serve_poll) with continuous
// batching.
//
// Requests carry a full problem (parameters, parareal configuration, host
// initial data).  Two lanes, each a scheduler thread that owns a batch
// (mm_batch.cpp) and a stream, run rounds: admit queued requests of the lane
// while their device footprint fits the HBM budget (shared by the lanes) and
// a slot is free, run one parareal iteration of every resident solve of the
// lane (the fine propagations of all of them share one persistent work-list
// launch), and hand out the solves that finished.  A request that arrives
// while others are on the GPU joins its lane at the next round; its result
// does not depend on which other solves it ran with.
//
// Lanes: a request whose parareal iteration costs more than kLongCost fine
// cell-updates (estimated from the step rule) goes to the long lane, every
// other one to the short lane.  The long lane's launches use at most
// n_sm - n_sm/8 CTAs, so one eighth of the SMs stays free for the short
// lane: a small request does not wait behind a round of large solves that
// takes seconds.  While the long lane has nothing resident, the short lane's
// launches may use every SM.
#include <math.h>
#include <string.h>

#include <atomic>
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

// fine cell-updates per parareal iteration above which a request is long
constexpr double kLongCost = 2e10;

struct Job {
  uint64_t ticket = 0;
  mm_params params{};
  mm_parareal_cfg cfg{};
  std::vector<double> rho0;
  std::vector<unsigned char> g0;
  size_t footprint = 0;
  int lane = 0;
  Clock::time_point t_submit;
  uint64_t batch_id = 0;
  // result
  bool done = false;
  mm_status status = MM_OK;
  std::vector<double> rho_T;
  int iterations = 0;
  int64_t latency_ns = 0;
  int64_t kinetic_updates = 0;
};

}  // namespace

struct mm_server {
  mm_server_cfg cfg{};
  mm_alloc alloc{};
  bool has_alloc = false;
  int device = 0;
  int n_sm = 1;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<std::shared_ptr<Job>> queue[2];       // per lane: 0 short, 1 long
  std::map<uint64_t, std::shared_ptr<Job>> jobs;  // by ticket, until polled
  size_t in_use = 0;
  int running = 0;
  std::atomic<int> long_resident{0};
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread sched[2];

  // device bytes a request holds while resident: its arrays plus its share
  // of the fine kernel's per-CTA step buffers (sized for the largest state)
  size_t footprint_of(const mm_params& p, const mm_parareal_cfg& c) const {
    const size_t gsz = p.precision == MM_FP32G ? 4 : 8;
    return mm_batch_footprint(&p, &c) + 2 * (size_t)p.nx * p.nv * gsz * n_sm + (1u << 20);
  }

  void finish(const std::shared_ptr<Job>& j, mm_status st) {
    std::lock_guard<std::mutex> lk(mu);
    j->status = st;
    j->latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - j->t_submit).count();
    j->done = true;
    in_use -= j->footprint;
    --running;
    if (j->lane == 1) --long_resident;
    cv_done.notify_all();
    cv_sched.notify_all();  // freed budget may admit a request of the other lane
  }

  void scheduler(int lane) {
    cudaSetDevice(device);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    mm_batch* batch = nullptr;
    mm_status bst = mm_batch_create(has_alloc ? &alloc : nullptr, &batch);
    const int reserve = n_sm >= 16 ? n_sm / 8 : 0;  // SMs kept for the short lane
    std::map<uint64_t, std::shared_ptr<Job>> inflight;  // by batch id
    while (true) {
      std::vector<std::shared_ptr<Job>> admit;
      {
        std::unique_lock<std::mutex> lk(mu);
        auto& q = queue[lane];
        cv_sched.wait(lk, [&] {
          return stop || !inflight.empty() ||
                 (!q.empty() && running < cfg.max_slots && in_use + q.front()->footprint <= cfg.hbm_budget_bytes);
        });
        if (stop) break;
        while (!q.empty() && running < cfg.max_slots && in_use + q.front()->footprint <= cfg.hbm_budget_bytes) {
          admit.push_back(q.front());
          in_use += q.front()->footprint;
          ++running;
          if (lane == 1) ++long_resident;
          q.pop_front();
        }
      }
      for (auto& j : admit) {
        if (bst != MM_OK) {
          finish(j, bst);
          continue;
        }
        mm_status st = mm_batch_add(batch, &j->params, &j->cfg, j->rho0.data(), j->g0.data(), &j->batch_id);
        if (st != MM_OK) finish(j, st);
        else inflight[j->batch_id] = j;
      }
      if (inflight.empty()) continue;
      if (bst == MM_OK) {
        mmk::batch_set_max_ctas(batch, lane == 1 ? n_sm - reserve : (long_resident.load() > 0 ? reserve : n_sm));
        mmk::batch_set_cluster_min_nx(batch, mmk::kServeClusterMinNx);
      }
      int32_t active = 0;
      mm_status st = mm_batch_step(batch, &active, s);
      if (st != MM_OK) {  // the round failed: every resident solve fails with it
        for (auto& kv : inflight) finish(kv.second, st);
        inflight.clear();
        mm_batch_destroy(batch);
        bst = mm_batch_create(has_alloc ? &alloc : nullptr, &batch);
        continue;
      }
      for (auto it = inflight.begin(); it != inflight.end();) {
        int32_t done = 0;
        mm_batch_query(batch, it->first, &done);
        if (!done) {
          ++it;
          continue;
        }
        auto j = it->second;
        std::vector<double> slices((size_t)(j->cfg.n_slices + 1) * j->params.nx);
        mm_parareal_stats ps{};
        const mm_status ts = mm_batch_take(batch, it->first, slices.data(), &ps);
        if (ts == MM_OK) {
          j->rho_T.assign(slices.end() - j->params.nx, slices.end());
          j->iterations = ps.iterations;
          j->kinetic_updates = ps.kinetic_updates;
        }
        finish(j, ts);
        it = inflight.erase(it);
      }
    }
    for (auto& kv : inflight) finish(kv.second, MM_ERR_INVALID);
    if (batch) mm_batch_destroy(batch);
    cudaStreamDestroy(s);
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
  cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, s->device);
  if (s->n_sm <= 0) s->n_sm = 1;
  for (int lane = 0; lane < 2; ++lane) s->sched[lane] = std::thread([s, lane] { s->scheduler(lane); });
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
  j->footprint = s->footprint_of(p, req->cfg);
  j->lane = mmk::solve_iteration_cost(p, req->cfg) > kLongCost ? 1 : 0;
  if (j->footprint > s->cfg.hbm_budget_bytes)
    return mm_fail(MM_ERR_INVALID, "request footprint exceeds the whole HBM budget");
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return mm_fail(MM_ERR_INVALID, "server is stopping");
  j->ticket = s->next_ticket++;
  s->jobs[j->ticket] = j;
  s->queue[j->lane].push_back(j);
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
  const int wait = std::min(std::max(0, (int)timeout_ms), s->cfg.wait_limit_ms);
  if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(wait), [&] { return j->done; }))
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
    for (auto& q : s->queue) {
      for (auto& j : q) {
        j->status = MM_ERR_INVALID;
        j->done = true;
      }
      q.clear();
    }
  }
  s->cv_sched.notify_all();
  for (auto& t : s->sched)
    if (t.joinable()) t.join();
  s->cv_done.notify_all();
  delete s;
  return MM_OK;
}
