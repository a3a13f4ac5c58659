// Batch engine: many parareal solves (Algorithm 1, Sec. 3.3) of different
// shapes advanced together, one parareal iteration of every unfinished solve
// per round.  A round is three launches whatever the number of solves:
//   - the coarse guess of the solves added since the last round (one CTA per
//     solve, sequential over its slices);
//   - the fine propagations of every (solve, slice) pair the iteration needs,
//     as one work list walked by the persistent fine kernel (one launch per
//     class of precision and adaptation), longest items first; each item
//     lifts its slice density in place, so no per-slice g is stored;
//   - the sequential corrections and successive errors (one CTA per solve).
// A solve leaves the batch when it reaches its iteration cap or its
// tolerance; new solves can be added between rounds (continuous batching).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <memory>
#include <vector>

#include "mm_internal.h"

namespace {

struct Solve {
  uint64_t id = 0;
  mm_ctx* ctx = nullptr;
  mm_parareal_cfg cfg{};
  int N = 0, K = 0, nx = 0, nv = 0, lanes = 0;
  bool fp32 = false, adapt = false;
  int64_t nf = 0;
  double dtf = 0, span = 0, rb = 0;
  double *rho = nullptr, *frho = nullptr, *gprev = nullptr;
  void* g0 = nullptr;
  size_t bytes = 0;
  int k = 0;
  bool started = false, done = false;
  std::vector<double> errs;
  int64_t kin = 0;
};

}  // namespace

struct mm_batch {
  mm_alloc cb{};
  bool has_cb = false;
  int device = 0;
  int n_sm = 0;
  int max_ctas = 0;  // cap on the work-list launch's CTAs (0: one per SM)
  int cluster_min_nx = 4096;  // sequential parts of solves from this grid on run over a cluster
  uint64_t next_id = 1;
  std::map<uint64_t, std::unique_ptr<Solve>> solves;
  size_t bytes_in_use = 0;
  // growable device buffers
  struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
  };
  Buf fine_ws, macro_ws, tables, items, corr, counters;
  double fine_ms = 0;
  int fine_launches = 0;
  int64_t kin_total = 0;

  void* dalloc(size_t bytes, cudaStream_t s) {
    void* p = nullptr;
    if (has_cb) return cb.alloc(bytes, s, cb.user);
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void dfree(void* p, cudaStream_t s) {
    if (!p) return;
    if (has_cb) cb.free(p, s, cb.user);
    else cudaFreeAsync(p, s);
  }
  mm_status grow(Buf& b, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return MM_OK;
    dfree(b.p, s);
    b.p = dalloc(bytes, s);
    b.bytes = b.p ? bytes : 0;
    return b.p ? MM_OK : mm_fail(MM_ERR_OOM, "batch: device allocation failed");
  }
  void release(Solve& v, cudaStream_t s) {
    dfree(v.rho, s);
    dfree(v.frho, s);
    dfree(v.gprev, s);
    dfree(v.g0, s);
    v.rho = v.frho = v.gprev = nullptr;
    v.g0 = nullptr;
    if (v.ctx) mmk::ctx_release(v.ctx, s);
    v.ctx = nullptr;
    bytes_in_use -= v.bytes;
  }
};

// device bytes a solve holds while resident in a batch
extern "C" size_t mm_batch_footprint(const mm_params* p, const mm_parareal_cfg* cfg) {
  if (!p || !cfg) return 0;
  const size_t gsz = p->precision == MM_FP32G ? 4 : 8;
  return 3 * (size_t)(cfg->n_slices + 1) * p->nx * 8 + (size_t)p->nx * p->nv * gsz;
}

extern "C" mm_status mm_batch_create(const mm_alloc* alloc, mm_batch** out) {
  if (!out) return mm_fail(MM_ERR_INVALID, "out is NULL");
  mm_batch* b = new mm_batch();
  if (alloc && alloc->alloc && alloc->free) {
    b->cb = *alloc;
    b->has_cb = true;
  }
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
  if (b->n_sm <= 0) b->n_sm = 1;
  *out = b;
  return MM_OK;
}

extern "C" mm_status mm_batch_add(mm_batch* b, const mm_params* p, const mm_parareal_cfg* cfg, const double* rho0,
                                  const void* g0, uint64_t* id) {
  if (!b || !p || !cfg || !rho0 || !g0 || !id) return mm_fail(MM_ERR_INVALID, "NULL argument");
  if (cfg->n_slices < 1 || cfg->max_iter < 0 || !(cfg->t_end > 0))
    return mm_fail(MM_ERR_INVALID, "bad parareal configuration");
  if (cfg->mode != MM_PARAREAL_RHO_LIFT)
    return mm_fail(MM_ERR_INVALID, "batch: only the density mode of Algorithm 1 (MM_PARAREAL_RHO_LIFT)");
  cudaSetDevice(b->device);
  std::unique_ptr<Solve> v(new Solve());
  mm_status st = mm_create(p, b->has_cb ? &b->cb : nullptr, &v->ctx);
  if (st != MM_OK) return st;
  if (!mmk::ctx_list_layout(v->ctx, &v->lanes)) {
    mmk::ctx_release(v->ctx, 0);
    return mm_fail(MM_ERR_INVALID, "batch: nv needs 8 velocity nodes per lane (FP32) or 4 (FP64)");
  }
  v->cfg = *cfg;
  v->N = cfg->n_slices;
  v->K = std::min(cfg->max_iter, cfg->n_slices);
  v->nx = p->nx;
  v->nv = p->nv;
  v->fp32 = p->precision == MM_FP32G;
  v->adapt = p->adapt != 0;
  v->span = cfg->t_end / v->N;
  v->nf = mmk::ctx_fine_steps(v->ctx, v->span);
  v->dtf = v->span / v->nf;
  const size_t rowb = (size_t)v->nx * 8, gb = (size_t)v->nx * v->nv * (v->fp32 ? 4 : 8);
  cudaStream_t s = 0;
  v->rho = (double*)b->dalloc(rowb * (v->N + 1), s);
  v->frho = (double*)b->dalloc(rowb * (v->N + 1), s);
  v->gprev = (double*)b->dalloc(rowb * (v->N + 1), s);
  v->g0 = b->dalloc(gb, s);
  v->bytes = mm_batch_footprint(p, cfg);
  b->bytes_in_use += v->bytes;
  if (!v->rho || !v->frho || !v->gprev || !v->g0) {
    b->release(*v, s);
    return mm_fail(MM_ERR_OOM, "batch: device allocation failed");
  }
  // rho_bar: the mean of the initial density when NaN
  std::vector<double> h(v->nx);
  cudaError_t e = cudaMemcpy(h.data(), rho0, rowb, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(v->rho, rho0, rowb, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(v->g0, g0, gb, cudaMemcpyDefault);
  if (e != cudaSuccess) {
    b->release(*v, s);
    return mm_cuda_fail(e, "batch: copying the initial data");
  }
  v->rb = isnan(p->rho_bar) ? mmk::ctx_mean(h.data(), v->nx) : p->rho_bar;
  v->id = b->next_id++;
  *id = v->id;
  b->solves[v->id] = std::move(v);
  return MM_OK;
}

// One parareal iteration of every unfinished solve.
// A solve's sequential parts (coarse guess, correction) run over a
// thread-block cluster, one cluster of 8 SMs per solve, from the batch's
// cluster_min_nx on, else on one CTA.  The one-CTA step is bound by its
// SM's FP64 pipe (about 0.3 ms per step at Nx = 8192, 0.7 ms at 32768), and
// the longest such chain sets the length of a step's correction launch; the
// cluster step shortens that chain several-fold (57 us against 0.7 ms at
// Nx = 32768) for 8 SMs per solve while it runs.  On small grids it costs
// far more SM time than one CTA (at Nx = 1024, 10.9 us on 8 SMs against
// 19 us on one).  A batch that shares the GPU with another (the server's two
// lanes) keeps the clusters for the largest grids: a cluster needs 8 free
// SMs of one GPC, which the other batch's launches may hold.
static bool on_cluster(const mmk::CorrectArgs& c, int min_nx) {
  return c.m.nx >= min_nx && mmk::coarse_cluster_ok(c.m);
}

// Orders `ca` for launch_sequential: the one-CTA entries first, then the
// cluster entries grouped by grid size; returns the one-CTA count.
static int order_sequential(std::vector<mmk::CorrectArgs>& ca, int min_nx) {
  std::stable_sort(ca.begin(), ca.end(), [min_nx](const mmk::CorrectArgs& x, const mmk::CorrectArgs& y) {
    return (on_cluster(x, min_nx) ? x.m.nx : 0) < (on_cluster(y, min_nx) ? y.m.nx : 0);
  });
  int n = 0;
  while (n < (int)ca.size() && !on_cluster(ca[n], min_nx)) ++n;
  return n;
}

// The coarse guesses (guess = true) or the corrections of the entries of
// `ca`, ordered by order_sequential and uploaded to d: one work-list launch
// of one CTA per solve, then one cluster launch per grid size.
static cudaError_t launch_sequential(const std::vector<mmk::CorrectArgs>& ca, const mmk::CorrectArgs* d,
                                     int n_small, bool guess, int nx_max, double* ws, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (n_small > 0)
    e = guess ? mmk::launch_coarse_chain_list(d, n_small, nx_max, ws, s)
              : mmk::launch_correct_list(d, n_small, nx_max, ws, s);
  for (int i = n_small; e == cudaSuccess && i < (int)ca.size();) {
    int j = i;
    while (j < (int)ca.size() && ca[j].m.nx == ca[i].m.nx) ++j;
    e = guess ? mmk::launch_coarse_chain_cluster_list(d + i, j - i, ca[i].m.nx, s)
              : mmk::launch_correct_cluster_list(d + i, j - i, ca[i].m.nx, s);
    i = j;
  }
  return e;
}

extern "C" mm_status mm_batch_step(mm_batch* b, int32_t* active_out, void* stream) {
  if (!b) return mm_fail(MM_ERR_INVALID, "batch is NULL");
  cudaSetDevice(b->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<Solve*> act, fresh;
  for (auto& kv : b->solves) {
    Solve* v = kv.second.get();
    if (v->done) continue;
    act.push_back(v);
    if (!v->started) fresh.push_back(v);
  }
  if (active_out) *active_out = (int32_t)act.size();
  if (act.empty()) return MM_OK;
  mm_status st;
  cudaError_t e;

  // ---- coarse guess of the new solves
  int nx_max = 0;
  for (Solve* v : act) nx_max = std::max(nx_max, v->nx);
  const int n_macro = (int)act.size();
  const size_t mws = mmk::macro_list_ws_bytes(nx_max, n_macro);
  if (mws && (st = b->grow(b->macro_ws, mws, s)) != MM_OK) return st;
  if ((st = b->grow(b->corr, sizeof(mmk::CorrectArgs) * n_macro + 8 * n_macro + 64, s)) != MM_OK) return st;
  mmk::CorrectArgs* d_corr = (mmk::CorrectArgs*)b->corr.p;
  double* d_err = (double*)((char*)b->corr.p + sizeof(mmk::CorrectArgs) * n_macro);
  std::vector<mmk::CorrectArgs> ca;
  if (!fresh.empty()) {
    for (Solve* v : fresh) {
      mmk::CorrectArgs c{};
      c.m = mmk::ctx_macro_args(v->ctx, v->span, v->rb);
      c.n_slices = v->N;
      c.rho = v->rho;
      c.gprev = v->gprev;
      ca.push_back(c);
      v->started = true;
    }
    const int n_small = order_sequential(ca, b->cluster_min_nx);
    e = cudaMemcpyAsync(d_corr, ca.data(), sizeof(mmk::CorrectArgs) * ca.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_sequential(ca, d_corr, n_small, true, nx_max, (double*)b->macro_ws.p, s);
    if (e != cudaSuccess) return mm_cuda_fail(e, "batch: coarse guess");
    // the argument table is reused below: the copy above must be consumed
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return mm_cuda_fail(e, "batch: coarse guess");
    // K = 0: the coarse guess is the result
    for (Solve* v : fresh)
      if (v->K == 0) v->done = true;
    act.erase(std::remove_if(act.begin(), act.end(), [](Solve* v) { return v->done; }), act.end());
    if (act.empty()) return MM_OK;
  }

  // ---- fine propagations: one work list per (precision, adaptation) class
  if ((st = b->grow(b->counters, 16 + 8 * act.size(), s)) != MM_OK) return st;
  unsigned long long* d_kin = (unsigned long long*)((char*)b->counters.p + 16);
  int* d_next = (int*)b->counters.p;
  int* d_status = (int*)b->counters.p + 1;
  e = cudaMemsetAsync(b->counters.p, 0, 16 + 8 * act.size(), s);
  if (e != cudaSuccess) return mm_cuda_fail(e, "batch: counters");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  for (int cls = 0; cls < 4; ++cls) {
    const bool fp32 = cls & 1, adapt = cls & 2;
    std::vector<mmk::FineListSolve> tab;
    std::vector<mmk::FineListItem> items;
    std::vector<double> cost;
    size_t ws_g = 16, ws_col = 16, smem_in = 0;
    for (size_t q = 0; q < act.size(); ++q) {
      Solve* v = act[q];
      if (v->fp32 != fp32 || v->adapt != adapt) continue;
      mmk::FineListSolve fs{};
      fs.a = mmk::ctx_fine_args(v->ctx, v->nf, v->dtf, v->rb);
      fs.a.kin_count = d_kin + q;
      fs.a.status = d_status;
      fs.rho = v->rho;
      fs.frho = v->frho;
      fs.g0 = v->k == 0 ? v->g0 : nullptr;
      const int si = (int)tab.size();
      tab.push_back(fs);
      for (int n = v->k; n < v->N; ++n) {
        items.push_back({si, n});
        cost.push_back((double)v->nf * v->nx * v->nv);
      }
      ws_g = std::max(ws_g, (size_t)v->nx * v->nv * (fp32 ? 4 : 8));
      ws_col = std::max(ws_col, mmk::fine_column_bytes(v->nx, v->nv, v->lanes, fp32, adapt, true));
      smem_in = std::max(smem_in, mmk::fine_smem_bytes(v->nx, v->nv, v->lanes, fp32, adapt, true));
    }
    if (items.empty()) continue;
    // longest first (dynamic scheduling of uneven items)
    std::vector<int> order(items.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<mmk::FineListItem> sorted(items.size());
    for (size_t q = 0; q < order.size(); ++q) sorted[q] = items[order[q]];
    ws_g = (ws_g + 255) & ~size_t(255);
    ws_col = (ws_col + 255) & ~size_t(255);
    const int cap = b->max_ctas > 0 ? std::min(b->max_ctas, b->n_sm) : b->n_sm;
    const int grid = (int)std::min<size_t>(sorted.size(), (size_t)cap);
    const size_t per_cta = 2 * ws_g + ws_col;
    if ((st = b->grow(b->fine_ws, per_cta * grid, s)) != MM_OK) return st;
    const size_t tb = sizeof(mmk::FineListSolve) * tab.size();
    if ((st = b->grow(b->tables, tb, s)) != MM_OK) return st;
    if ((st = b->grow(b->items, sizeof(mmk::FineListItem) * sorted.size(), s)) != MM_OK) return st;
    e = cudaMemcpyAsync(b->tables.p, tab.data(), tb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->items.p, sorted.data(), sizeof(mmk::FineListItem) * sorted.size(),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_next, 0, sizeof(int), s);
    if (e != cudaSuccess) return mm_cuda_fail(e, "batch: work list upload");
    mmk::FineList L{};
    L.solves = (const mmk::FineListSolve*)b->tables.p;
    L.items = (const mmk::FineListItem*)b->items.p;
    L.n_items = (int)sorted.size();
    L.grid = grid;
    L.next = d_next;
    L.ws = (unsigned char*)b->fine_ws.p;
    L.ws_g = ws_g;
    L.ws_col = ws_col;
    e = mmk::launch_fine_list(L, fp32, adapt, smem_in, s);
    if (e != cudaSuccess) return mm_cuda_fail(e, "batch: fine work list launch");
    ++b->fine_launches;
    // the host tables are reused by the next class: wait for this launch's
    // uploads to be consumed
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return mm_cuda_fail(e, "batch: fine work list");
  }
  cudaEventRecord(e1, s);

  // ---- corrections and successive errors
  ca.clear();
  for (size_t q = 0; q < act.size(); ++q) {
    Solve* v = act[q];
    mmk::CorrectArgs c{};
    c.m = mmk::ctx_macro_args(v->ctx, v->span, v->rb);
    c.n_slices = v->N;
    c.k = v->k;
    c.rho = v->rho;
    c.frho = v->frho;
    c.gprev = v->gprev;
    c.err = d_err + q;
    ca.push_back(c);
  }
  const int n_small = order_sequential(ca, b->cluster_min_nx);
  e = cudaMemcpyAsync(d_corr, ca.data(), sizeof(mmk::CorrectArgs) * ca.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_sequential(ca, d_corr, n_small, false, nx_max, (double*)b->macro_ws.p, s);
  if (e != cudaSuccess) return mm_cuda_fail(e, "batch: corrections");
  std::vector<double> errs(act.size());
  std::vector<unsigned long long> kin(act.size());
  int hstat = 0;
  e = cudaMemcpyAsync(errs.data(), d_err, 8 * act.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(kin.data(), d_kin, 8 * act.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hstat, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return mm_cuda_fail(e, "batch: reading errors");
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->fine_ms += ms;
  for (size_t q = 0; q < act.size(); ++q) {
    Solve* v = act[q];
    v->errs.push_back(errs[q]);
    v->kin += (int64_t)kin[q];
    b->kin_total += (int64_t)kin[q];
    ++v->k;
    if (v->k >= v->K || errs[q] < v->cfg.tol) v->done = true;
  }
  if (hstat != 0) return mm_fail((mm_status)hstat, "batch: non-finite density in a fine propagation");
  return MM_OK;
}

extern "C" mm_status mm_batch_query(mm_batch* b, uint64_t id, int32_t* done) {
  if (!b || !done) return mm_fail(MM_ERR_INVALID, "NULL argument");
  auto it = b->solves.find(id);
  if (it == b->solves.end()) return mm_fail(MM_ERR_UNKNOWN_TICKET, "unknown solve id");
  *done = it->second->done ? 1 : 0;
  return MM_OK;
}

extern "C" mm_status mm_batch_take(mm_batch* b, uint64_t id, double* rho_slices_out, mm_parareal_stats* stats) {
  if (!b) return mm_fail(MM_ERR_INVALID, "batch is NULL");
  auto it = b->solves.find(id);
  if (it == b->solves.end()) return mm_fail(MM_ERR_UNKNOWN_TICKET, "unknown solve id");
  Solve& v = *it->second;
  if (!v.done) return mm_fail(MM_ERR_NOT_READY, "solve not finished");
  cudaSetDevice(b->device);
  const size_t bytes = (size_t)(v.N + 1) * v.nx * 8;
  std::vector<double> h((size_t)(v.N + 1) * v.nx);
  cudaError_t e = cudaMemcpy(h.data(), v.rho, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && rho_slices_out) e = cudaMemcpy(rho_slices_out, h.data(), bytes, cudaMemcpyDefault);
  if (e != cudaSuccess) return mm_cuda_fail(e, "batch: reading the result");
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iterations = (int32_t)v.errs.size();
    for (size_t q = 0; q < v.errs.size() && q < 64; ++q) stats->err[q] = v.errs[q];
    double m0 = 0;
    for (int i = 0; i < v.nx; ++i) m0 += h[i];
    double drift = 0;
    for (int n = 1; n <= v.N; ++n) {
      double m = 0;
      for (int i = 0; i < v.nx; ++i) m += h[(size_t)n * v.nx + i];
      drift = std::max(drift, fabs(m - m0) / fabs(m0));
    }
    stats->mass_drift = drift;
    stats->fine_steps = v.nf;
    stats->kinetic_updates = v.kin;
    stats->fine_ms = b->fine_ms;
    stats->fine_launches = b->fine_launches;
    stats->kernel_launches = 0;  // the engine's launches serve many solves (mm_batch_counters)
  }
  b->release(v, 0);
  b->solves.erase(it);
  return MM_OK;
}

extern "C" void mm_batch_destroy(mm_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  for (auto& kv : b->solves) b->release(*kv.second, 0);
  b->dfree(b->fine_ws.p, 0);
  b->dfree(b->macro_ws.p, 0);
  b->dfree(b->tables.p, 0);
  b->dfree(b->items.p, 0);
  b->dfree(b->corr.p, 0);
  b->dfree(b->counters.p, 0);
  cudaStreamSynchronize(0);
  delete b;
}

extern "C" size_t mm_batch_bytes(const mm_batch* b) { return b ? b->bytes_in_use : 0; }

extern "C" mm_status mm_batch_counters(const mm_batch* b, int64_t* kinetic_updates, int32_t* fine_launches,
                                       double* fine_ms) {
  if (!b) return mm_fail(MM_ERR_INVALID, "batch is NULL");
  if (kinetic_updates) *kinetic_updates = b->kin_total;
  if (fine_launches) *fine_launches = b->fine_launches;
  if (fine_ms) *fine_ms = b->fine_ms;
  return MM_OK;
}

extern "C" mm_status parareal_run_many(int32_t n, const mm_params* params, const mm_parareal_cfg* cfgs,
                                       const double* const* rho0, const void* const* g0,
                                       double* const* rho_slices_out, mm_parareal_stats* stats, void* stream) {
  if (n < 0 || (n > 0 && (!params || !cfgs || !rho0 || !g0 || !rho_slices_out)))
    return mm_fail(MM_ERR_INVALID, "bad arguments");
  if (n == 0) return MM_OK;
  mm_batch* b = nullptr;
  mm_status st = mm_batch_create(nullptr, &b);
  if (st != MM_OK) return st;
  std::vector<uint64_t> ids(n);
  for (int q = 0; q < n && st == MM_OK; ++q) st = mm_batch_add(b, params + q, cfgs + q, rho0[q], g0[q], &ids[q]);
  int32_t active = 1;
  while (st == MM_OK && active > 0) st = mm_batch_step(b, &active, stream);
  for (int q = 0; q < n && st == MM_OK; ++q)
    st = mm_batch_take(b, ids[q], rho_slices_out[q], stats ? stats + q : nullptr);
  mm_batch_destroy(b);
  return st;
}

void mmk::batch_set_max_ctas(mm_batch* b, int n) {
  if (b) b->max_ctas = n > 0 ? n : 0;
}

void mmk::batch_set_cluster_min_nx(mm_batch* b, int nx) {
  if (b) b->cluster_min_nx = nx;
}
