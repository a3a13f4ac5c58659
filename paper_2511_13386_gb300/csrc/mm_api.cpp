// Host side of the C ABI declared in include/mm.h: contexts, parameter
// validation, the step-size rule, staging of host arrays, the fine / coarse
// / lift entry points and the parareal driver of Algorithm 1 (Sec. 3.3).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "mm_internal.h"

// ------------------------------------------------------------- errors ---

static thread_local std::string g_last_error;

mm_status mm_fail(mm_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

mm_status mm_cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA;
}

extern "C" const char* mm_last_error(void) { return g_last_error.c_str(); }

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return mm_cuda_fail(e_, what); \
  } while (0)

// ----------------------------------------------------------- workspace --

namespace {

// Named device buffers grown on demand; memory from the user's callbacks or
// from the stream-ordered allocator.
struct Workspace {
  mm_alloc cb{};
  bool has_cb = false;
  struct Slot {
    void* p = nullptr;
    size_t bytes = 0;
  };
  std::vector<Slot> slots;

  void release(Slot& s, cudaStream_t st) {
    if (!s.p) return;
    if (has_cb) cb.free(s.p, st, cb.user);
    else cudaFreeAsync(s.p, st);
    s.p = nullptr;
    s.bytes = 0;
  }

  mm_status get(int id, size_t bytes, cudaStream_t st, void** out) {
    if ((int)slots.size() <= id) slots.resize(id + 1);
    Slot& s = slots[id];
    if (bytes == 0) bytes = 16;
    if (s.bytes < bytes) {
      release(s, st);
      void* p = nullptr;
      if (has_cb) {
        p = cb.alloc(bytes, st, cb.user);
        if (!p) return mm_fail(MM_ERR_OOM, "workspace allocation failed (callback)");
      } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, st);
        if (e != cudaSuccess) return mm_cuda_fail(e, "cudaMallocAsync(workspace)");
      }
      s.p = p;
      s.bytes = bytes;
    }
    *out = s.p;
    return MM_OK;
  }

  void release_all(cudaStream_t st) {
    for (auto& s : slots) release(s, st);
  }
};

// A pair of timing events, released on every return path.
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  explicit EventPair(bool on) {
    if (on) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
    }
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  EventPair(const EventPair&) = delete;
  EventPair& operator=(const EventPair&) = delete;
};

enum WsSlot {
  WS_GBUF1 = 0, WS_COLS, WS_RHO_IN, WS_RHO_OUT, WS_G_IN, WS_G_OUT, WS_MASK, WS_MACRO,
  WS_STATUS, WS_PR_RHO, WS_PR_F, WS_PR_G, WS_PR_GB, WS_PR_ERR, WS_PR_GB2, WS_PR_GOLD, WS_PR_LD, WS_PR_SUM,
  WS_COUNT
};

}  // namespace

struct mm_ctx {
  mm_params p{};
  int device = 0;
  mmk::VelocityGrid vg;
  mmk::LaneLayout lay;       // default streaming layout (the batch engine's)
  mmk::LaneLayout fine_lay;  // streaming layout of mm_fine_propagate (params.fine_vpt)
  double dt_rule = 0;     // stability limit of the rule at cfl_theta
  double dt_limit = 0;    // limit actually used (params.dt or dt_rule)
  double* d_vtab = nullptr;
  float* d_vtab_f = nullptr;
  Workspace ws;
  // launch shape of F chosen by mm_autotune (tuned == 0: the defaults)
  int tuned = 0;
  int tuned_kernel = 0;       // 1 streaming, 2 resident
  int tuned_cluster = 0;      // resident: CTAs per state
  mmk::LaneLayout tuned_lay;  // streaming: lane layout
  double res_entry = 0;       // resident: measured chunk entry cost (step-equivalents; 0: estimate)
  // second stream and events of parareal_run's overlap of Algorithm 1's
  // sequential parts with the resident kernel's rounds (created on first use)
  cudaStream_t side = nullptr;
  cudaEvent_t ov[4] = {nullptr, nullptr, nullptr, nullptr};
};

// ------------------------------------------------------- launch choice ---

namespace {
struct FineChoice {
  int kernel = 1;          // 1 streaming, 2 resident
  int C = 0;               // resident cluster size
  size_t res_smem = 0;
  mmk::LaneLayout lay;     // streaming lane layout
};
}  // namespace

// The F implementation and launch shape mm_fine_propagate uses: the tuned
// one, else the resident kernel whenever the shape allows it (unless
// params.fine_kernel asks for the streaming one), with the default lane
// layout for the streaming kernel.
static FineChoice fine_choice(const mm_ctx* c) {
  const mm_params& p = c->p;
  const bool fp32 = p.precision == MM_FP32G, adapt = p.adapt != 0;
  FineChoice f;
  f.lay = c->fine_lay;
  if (c->tuned) {
    f.kernel = c->tuned_kernel;
    if (f.kernel == 2) {
      f.C = c->tuned_cluster;
      f.res_smem = mmk::fine_resident_smem(p.nx, p.nv, fp32, adapt, p.flux_rule, f.C);
    } else {
      f.lay = c->tuned_lay;
    }
    return f;
  }
  if (p.fine_kernel != 1) f.C = mmk::fine_resident_cluster(p.nx, p.nv, fp32, adapt, p.flux_rule, &f.res_smem);
  f.kernel = f.C ? 2 : 1;
  return f;
}

// ----------------------------------------------------------- parameters --

extern "C" void mm_params_default(mm_params* p) {
  memset(p, 0, sizeof(*p));
  p->nx = 64;
  p->nv = 32;
  p->x_len = 1.0;
  p->v_max = 8.0;
  p->eps = 1.0;
  p->rho_bar = NAN;
  p->adapt = 0;
  p->thr_g = 1e-3;
  p->thr_R = 1e-2;
  p->r_scale = 0;
  p->flux_rule = 0;
  p->dt = 0.0;
  p->cfl_theta = 0.9;
  p->coarse_kind = 0;
  p->coarse_steps = 1;
  p->lift_order = 1;
  p->precision = MM_FP64;
}

// Velocity discretisation of Sec. 2.3 with trapezoid weights and the
// Maxwellian normalised on the grid.
static mmk::VelocityGrid build_velocity_grid(int nv, double v_max) {
  mmk::VelocityGrid g;
  g.nv = nv;
  g.dv = 2.0 * v_max / (nv - 1);
  g.v.resize(nv);
  g.w.resize(nv);
  g.M.resize(nv);
  double Z = 0.0;
  for (int j = 0; j < nv; ++j) {
    g.v[j] = (double)(2 * j - nv + 1) * (0.5 * g.dv);
    g.w[j] = (j == 0 || j == nv - 1) ? 0.5 * g.dv : g.dv;
    Z += g.w[j] * exp(-0.5 * g.v[j] * g.v[j]);
  }
  g.m2 = 0.0;
  g.xiM = 0.0;
  g.mu3 = 0.0;
  for (int j = 0; j < nv; ++j) {
    g.M[j] = exp(-0.5 * g.v[j] * g.v[j]) / Z;
    g.m2 += g.w[j] * g.v[j] * g.v[j] * g.M[j];
    g.xiM += g.w[j] * g.v[j] * g.M[j];
    g.mu3 += g.w[j] * g.v[j] * g.v[j] * g.v[j] * g.M[j];
  }
  return g;
}

// Stability rule for the step (the paper states none).  With
// a(s) = exp(-s/eps^2), phi_t = 2 eps (1-a) v_max / (dx (1+a)) (upwind
// transport of g with relaxation) and phi_d = 2 m2 s (1-a) / dx^2
// (diffusion of rho through g), the step s must satisfy phi_t <= 1,
// phi_d <= 1, phi_d + phi_t / 4 <= 1 (the two couple: a von Neumann
// analysis of the linearised step puts the critical phi_d near
// 1 - 0.21 phi_t in the diffusive regime) and, with adaptation, the explicit
// S^0 limit 2 m2 s / dx^2 <= 1 in fluid cells; the largest such s is
// bracketed and bisected.
static bool step_ok(const mm_params& p, double m2, double s) {
  const double dx = p.x_len / p.nx;
  const double a = exp(-s / (p.eps * p.eps));
  const double phi_t = 2.0 * p.eps * (1.0 - a) * p.v_max / (dx * (1.0 + a));
  const double phi_d = 2.0 * m2 * s * (1.0 - a) / (dx * dx);
  if (phi_t > 1.0 || phi_d > 1.0 || phi_d + 0.25 * phi_t > 1.0) return false;
  if (p.adapt && 2.0 * m2 * s / (dx * dx) > 1.0) return false;
  return true;
}

static double stability_limit(const mm_params& p, double m2) {
  double lo = 0.0, hi = 1.0;
  while (step_ok(p, m2, hi) && hi < 1e300) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (step_ok(p, m2, mid)) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Lane layout of the streaming kernel with vpt velocity nodes per lane:
// each half of the velocity grid gets nh = nv / 2 / vpt lanes, padded to a
// power of two; at most 32 lanes per column.
static bool layout_for(int nv, int vpt, mmk::LaneLayout* out) {
  if (nv < 4 || nv % 2 || (nv / 2) % vpt) return false;
  const int nh = nv / 2 / vpt;
  int nhp = 1;
  while (nhp < nh) nhp <<= 1;
  if (2 * nhp > 32) return false;
  out->vpt = vpt;
  out->nh = nh;
  out->nhp = nhp;
  out->lanes = 2 * nhp;
  return true;
}

static const int kVpt32[] = {8, 4, 2, 1}, kVpt64[] = {4, 2, 1, 8};

// Whether the streaming kernel offers vpt nodes per lane for this nv and
// precision.  FP64 takes 8 nodes per lane only where 4 would need more than
// 32 lanes (nv = 256): 8 doubles per lane cost registers the other layouts
// keep.
static bool vpt_offered(int nv, bool fp32, int vpt, mmk::LaneLayout* out) {
  mmk::LaneLayout l4;
  if (!fp32 && vpt == 8 && layout_for(nv, 4, &l4)) return false;
  return layout_for(nv, vpt, out);
}

// Default layout: the most velocity nodes per lane that works.
static bool choose_layout(int nv, bool fp32, mmk::LaneLayout* out) {
  const int* c = fp32 ? kVpt32 : kVpt64;
  for (int q = 0; q < 4; ++q)
    if (vpt_offered(nv, fp32, c[q], out)) return true;
  return false;
}

static mm_status validate(const mm_params* p) {
  if (!p) return mm_fail(MM_ERR_INVALID, "params is NULL");
  if (p->nx < 8 || p->nx > 65536) return mm_fail(MM_ERR_INVALID, "nx must be in [8, 65536]");
  if (p->nv < 4 || p->nv % 2) return mm_fail(MM_ERR_INVALID, "nv must be even and >= 4");
  if (!(p->x_len > 0) || !(p->v_max > 0) || !(p->eps > 0))
    return mm_fail(MM_ERR_INVALID, "x_len, v_max and eps must be positive");
  if (p->precision != MM_FP64 && p->precision != MM_FP32G)
    return mm_fail(MM_ERR_INVALID, "unknown precision");
  if (p->coarse_kind != 0 && p->coarse_kind != 1) return mm_fail(MM_ERR_INVALID, "coarse_kind must be 0 or 1");
  if (p->coarse_steps < 1) return mm_fail(MM_ERR_INVALID, "coarse_steps must be >= 1");
  if (p->lift_order < 1 || p->lift_order > 3) return mm_fail(MM_ERR_INVALID, "lift_order must be 1, 2 or 3");
  if (p->flux_rule != 0 && p->flux_rule != 1) return mm_fail(MM_ERR_INVALID, "flux_rule must be 0 or 1");
  if (p->dt < 0 || !(p->cfl_theta >= 0)) return mm_fail(MM_ERR_INVALID, "dt and cfl_theta must be >= 0");
  if (p->adapt && (!(p->thr_g >= 0) || !(p->thr_R >= 0)))
    return mm_fail(MM_ERR_INVALID, "thresholds must be >= 0");
  if (p->fine_kernel < 0 || p->fine_kernel > 2) return mm_fail(MM_ERR_INVALID, "fine_kernel must be 0, 1 or 2");
  if (p->fine_vpt != 0) {
    mmk::LaneLayout l;
    if (p->fine_vpt < 0 || p->fine_vpt > 8 || (p->fine_vpt & (p->fine_vpt - 1)) ||
        !vpt_offered(p->nv, p->precision == MM_FP32G, p->fine_vpt, &l))
      return mm_fail(MM_ERR_INVALID, "fine_vpt: no lane layout with that many nodes per lane for this nv");
  }
  if (p->fine_kernel == 2) {
    size_t sm;
    if (!mmk::fine_resident_cluster(p->nx, p->nv, p->precision == MM_FP32G, p->adapt != 0, p->flux_rule, &sm))
      return mm_fail(MM_ERR_INVALID, "fine_kernel 2 (resident) does not support this shape or option set");
  }
  return MM_OK;
}

extern "C" mm_status mm_create(const mm_params* p, const mm_alloc* alloc, mm_ctx** out) {
  if (!out) return mm_fail(MM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  mm_status st = validate(p);
  if (st != MM_OK) return st;
  mmk::LaneLayout lay;
  const bool fp32 = p->precision == MM_FP32G;
  if (!choose_layout(p->nv, fp32, &lay))
    return mm_fail(MM_ERR_INVALID,
                   "unsupported nv: nv/2 needs a divisor d in {1,2,4,8} with nv/d <= 32 lanes");
  mm_ctx* c = new mm_ctx();
  c->p = *p;
  if (c->p.cfl_theta == 0) c->p.cfl_theta = 0.9;
  c->lay = lay;
  c->fine_lay = lay;
  if (p->fine_vpt) layout_for(p->nv, p->fine_vpt, &c->fine_lay);
  if (alloc && alloc->alloc && alloc->free) {
    c->ws.cb = *alloc;
    c->ws.has_cb = true;
  }
  cudaGetDevice(&c->device);
  c->vg = build_velocity_grid(p->nv, p->v_max);
  c->dt_rule = c->p.cfl_theta * stability_limit(c->p, c->vg.m2);
  c->dt_limit = c->p.dt > 0 ? c->p.dt : c->dt_rule;

  const int nv = p->nv;
  const double dx = p->x_len / p->nx;
  std::vector<double> tab(mmk::kVTabFields * nv);
  for (int j = 0; j < nv; ++j) {
    const double v = c->vg.v[j], w = c->vg.w[j], M = c->vg.M[j];
    tab[0 * nv + j] = fabs(v) / dx;
    tab[1 * nv + j] = M;
    tab[2 * nv + j] = v * M;
    tab[3 * nv + j] = w * v;
    tab[4 * nv + j] = w;
    tab[5 * nv + j] = v;
  }
  std::vector<float> tabf(tab.begin(), tab.end());
  // stream-ordered allocation on the legacy stream: no device-wide
  // synchronisation, so contexts can come and go while other streams run
  cudaError_t e = cudaMallocAsync(&c->d_vtab, tab.size() * sizeof(double), 0);
  if (e == cudaSuccess) e = cudaMallocAsync(&c->d_vtab_f, tabf.size() * sizeof(float), 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_vtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_vtab_f, tabf.data(), tabf.size() * sizeof(float), cudaMemcpyHostToDevice, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) {
    if (c->d_vtab) cudaFreeAsync(c->d_vtab, 0);
    if (c->d_vtab_f) cudaFreeAsync(c->d_vtab_f, 0);
    cudaStreamSynchronize(0);
    delete c;
    return mm_cuda_fail(e, "mm_create: velocity table");
  }
  // everything mm_fine_propagate_noalloc needs from the device is reserved
  // here, so that its calls allocate nothing
  if ((st = mmk::noalloc_setup(c)) != MM_OK) {
    mmk::ctx_release(c, 0);
    cudaStreamSynchronize(0);
    return st;
  }
  *out = c;
  return MM_OK;
}

extern "C" void mm_destroy(mm_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  mmk::ctx_release(c, 0);
  cudaStreamSynchronize(0);
}

// Free a context's device memory in stream order on s, without a
// device-wide synchronisation (the batch engine: its solves' contexts have
// no work in flight once the batch's stream is synchronised, while another
// batch may be running on another stream).
void mmk::ctx_release(mm_ctx* c, cudaStream_t s) {
  if (!c) return;
  cudaSetDevice(c->device);
  c->ws.release_all(s);
  for (cudaEvent_t& ev : c->ov)
    if (ev) cudaEventDestroy(ev);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->d_vtab) cudaFreeAsync(c->d_vtab, s);
  if (c->d_vtab_f) cudaFreeAsync(c->d_vtab_f, s);
  delete c;
}

static int64_t steps_for(double span, double lim) {
  const double q = span / lim;
  int64_t n = (int64_t)ceil(q);
  return n < 1 ? 1 : n;
}

extern "C" mm_status mm_query(const mm_ctx* c, double t_span, mm_info* out) {
  if (!c || !out) return mm_fail(MM_ERR_INVALID, "NULL argument");
  if (!(t_span > 0)) return mm_fail(MM_ERR_INVALID, "t_span must be > 0");
  out->dt_limit = c->dt_limit;
  out->n_steps = steps_for(t_span, c->dt_limit);
  out->dt = t_span / out->n_steps;
  out->m2 = c->vg.m2;
  out->a = exp(-out->dt / (c->p.eps * c->p.eps));
  out->b = c->p.eps * (1.0 - out->a);
  const size_t gsz = c->p.precision == MM_FP32G ? 4 : 8;
  out->state_bytes = (size_t)c->p.nx * 8 + (size_t)c->p.nx * c->p.nv * gsz;
  const FineChoice f = fine_choice(c);
  out->vpt = f.lay.vpt;
  out->lanes = f.lay.lanes;
  out->fine_kernel = f.kernel;
  out->cluster = f.kernel == 2 ? f.C : 1;
  return MM_OK;
}

// --------------------------------------------------------- pointer kinds --

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device view of a caller array: the pointer itself, or a staging buffer
// (filled from the host when `copy_in`).
static mm_status device_view(mm_ctx* c, int slot, const void* p, size_t bytes, bool copy_in,
                             cudaStream_t s, void** out, bool* staged) {
  if (is_device_ptr(p) && ((uintptr_t)p % 16 == 0)) {
    *out = const_cast<void*>(p);
    *staged = false;
    return MM_OK;
  }
  mm_status st = c->ws.get(slot, bytes, s, out);
  if (st != MM_OK) return st;
  *staged = true;
  if (copy_in) CK(cudaMemcpyAsync(*out, p, bytes, cudaMemcpyDefault, s), "copy to device");
  return MM_OK;
}

// ----------------------------------------------------------- fine (F) ---

// Deferred completion of a fine call made by a driver that synchronises
// later anyway (parareal_run): the call records the caller's timing events
// around its launches and leaves its status word and kinetic-update counter
// on the device, instead of waiting for the launches to end.  Waiting there
// would hold back whatever the driver enqueues next on another stream to
// run beside the last launches (the correction of the slices already final).
struct FineDefer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;  // recorded around the launches (nullable)
  void* status = nullptr;                   // device: int status, ..., u64 counter at byte 16
  int launches = 0;
};

static mm_status fine_impl(mm_ctx* c, int32_t batch, int64_t n, double dt, const double* rho_in,
                           const void* g_in, double* rho_out, void* g_out, uint8_t* mask_out,
                           double rho_bar, mm_fine_stats* stats, cudaStream_t s,
                           const mmk::ResHooks* hooks = nullptr, FineDefer* defer = nullptr) {
  const mm_params& p = c->p;
  const bool fp32 = p.precision == MM_FP32G;
  const size_t gsz = fp32 ? 4 : 8;
  const size_t nx = p.nx, nv = p.nv;
  const size_t rbytes = batch * nx * 8, gbytes = batch * nx * nv * gsz, mbytes = batch * nx;

  void *d_rin, *d_gin, *d_rout, *d_gout, *d_mask = nullptr;
  bool s_rin, s_gin, s_rout, s_gout, s_mask = false;
  mm_status st;
  if ((st = device_view(c, WS_RHO_IN, rho_in, rbytes, true, s, &d_rin, &s_rin)) != MM_OK) return st;
  if ((st = device_view(c, WS_G_IN, g_in, gbytes, true, s, &d_gin, &s_gin)) != MM_OK) return st;
  if ((st = device_view(c, WS_RHO_OUT, rho_out, rbytes, false, s, &d_rout, &s_rout)) != MM_OK) return st;
  if ((st = device_view(c, WS_G_OUT, g_out, gbytes, false, s, &d_gout, &s_gout)) != MM_OK) return st;
  if (mask_out && (st = device_view(c, WS_MASK, mask_out, mbytes, false, s, &d_mask, &s_mask)) != MM_OK)
    return st;

  const bool adapt = p.adapt != 0;
  const FineChoice fc = fine_choice(c);
  const size_t res_smem = fc.res_smem;
  const int res_C = fc.kernel == 2 ? fc.C : 0;

  void* buf1 = nullptr;
  if (!res_C && (st = c->ws.get(WS_GBUF1, gbytes, s, &buf1)) != MM_OK) return st;
  // g_out is the buffer the last step writes; with an odd step count the
  // first step writes it too, so an aliased input is moved aside first.
  if (!res_C && d_gin == d_gout && (n & 1)) {
    CK(cudaMemcpyAsync(buf1, d_gin, gbytes, cudaMemcpyDeviceToDevice, s), "alias copy");
    d_gin = buf1;
    void* other;
    if ((st = c->ws.get(WS_G_IN, gbytes, s, &other)) != MM_OK) return st;
    buf1 = other;
  }

  mmk::FineArgs a{};
  a.nx = p.nx;
  a.nv = p.nv;
  a.batch = batch;
  a.n_steps = n;
  a.lanes = fc.lay.lanes;
  a.nh = fc.lay.nh;
  a.nhp = fc.lay.nhp;
  a.dt = dt;
  a.dx = p.x_len / p.nx;
  a.inv_dx = 1.0 / a.dx;
  a.inv_dv = 1.0 / c->vg.dv;
  a.eps = p.eps;
  a.inv_eps = 1.0 / p.eps;
  a.a = exp(-dt / (p.eps * p.eps));
  a.b = p.eps * (1.0 - a.a);
  a.m2 = c->vg.m2;
  a.dt_dx = dt / a.dx;
  a.rho_bar = rho_bar;
  a.adapt = p.adapt;
  a.r_scale = p.r_scale;
  a.flux_rule = p.flux_rule;
  a.thr_g = p.thr_g;
  a.thr_R = p.thr_R;
  a.r_fac = p.r_scale ? p.eps * p.eps : 1.0;
  a.rho_in = (const double*)d_rin;
  a.rho_out = (double*)d_rout;
  a.g_in = d_gin;
  a.g_buf0 = d_gout;
  a.g_buf1 = buf1;
  a.mask_out = (uint8_t*)d_mask;
  a.vtab = c->d_vtab;
  a.vtab_f = c->d_vtab_f;
  a.xiM = c->vg.xiM;
  a.mu3 = c->vg.mu3;
  a.lift_order = c->p.lift_order;
  a.res_entry_steps = c->res_entry;

  const size_t colb = mmk::fine_column_bytes(p.nx, p.nv, fc.lay.lanes, fp32, adapt, false);
  const bool in_smem = colb == 0;
  a.col_in_smem = in_smem ? 1 : 0;
  if (!in_smem && !res_C) {
    if ((st = c->ws.get(WS_COLS, colb * batch, s, &a.col_ws)) != MM_OK) return st;
    a.col_ws_stride = colb;
  }
  void* stat_mem;
  if ((st = c->ws.get(WS_STATUS, 64, s, &stat_mem)) != MM_OK) return st;
  a.status = (int*)stat_mem;
  a.kin_count = (unsigned long long*)((char*)stat_mem + 16);
  CK(cudaMemsetAsync(stat_mem, 0, 64, s), "memset status");

  EventPair ev(stats != nullptr && !defer);
  cudaEvent_t e0 = defer ? defer->e0 : ev.a, e1 = defer ? defer->e1 : ev.b;
  if (e0) cudaEventRecord(e0, s);
  const size_t smem = mmk::fine_smem_bytes(p.nx, p.nv, fc.lay.lanes, fp32, adapt, false);
  int launches = 1;
  cudaError_t e = res_C ? mmk::launch_fine_resident(a, res_C, res_smem, s, &launches, hooks)
                        : mmk::launch_fine(a, fc.lay.vpt, fp32, smem, s);
  if (e != cudaSuccess) return mm_cuda_fail(e, "fine kernel launch");
  if (e1) cudaEventRecord(e1, s);

  if (s_rout) CK(cudaMemcpyAsync(rho_out, d_rout, rbytes, cudaMemcpyDefault, s), "copy rho_out");
  if (s_gout) CK(cudaMemcpyAsync(g_out, d_gout, gbytes, cudaMemcpyDefault, s), "copy g_out");
  if (s_mask) CK(cudaMemcpyAsync(mask_out, d_mask, mbytes, cudaMemcpyDefault, s), "copy mask");

  if (defer) {  // the caller reads the status after its own synchronisation
    defer->status = stat_mem;
    defer->launches = launches;
    return MM_OK;
  }
  const bool host_out = s_rout || s_gout || s_mask;
  if (stats || host_out) {
    int hs[6] = {0};
    CK(cudaMemcpyAsync(hs, stat_mem, 24, cudaMemcpyDeviceToHost, s), "read status");
    CK(cudaStreamSynchronize(s), "fine: synchronise");
    if (stats) {
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      unsigned long long kc;
      memcpy(&kc, (char*)hs + 16, 8);
      stats->steps = n;
      stats->kinetic_updates = (int64_t)kc;
      stats->full_updates = (int64_t)n * batch * p.nx * p.nv;
      stats->device_status = hs[0];
      stats->elapsed_ms = ms;
      stats->launches = launches;
    }
    if (hs[0] != 0) return mm_fail((mm_status)hs[0], "fine: non-finite density");
  }
  return MM_OK;
}

static double stability_guard(const mm_ctx* c) {
  mm_params q = c->p;
  return stability_limit(q, c->vg.m2);
}

extern "C" mm_status mm_fine_propagate(mm_ctx* c, int32_t batch, double t_span, const double* rho_in,
                                       const void* g_in, double* rho_out, void* g_out, uint8_t* mask_out,
                                       mm_fine_stats* stats, void* stream) {
  if (!c) return mm_fail(MM_ERR_INVALID, "ctx is NULL");
  if (batch < 0) return mm_fail(MM_ERR_INVALID, "batch must be >= 0");
  if (!(t_span > 0)) return mm_fail(MM_ERR_INVALID, "t_span must be > 0");
  if (batch == 0) {
    if (stats) memset(stats, 0, sizeof(*stats));
    return MM_OK;
  }
  if (!rho_in || !g_in || !rho_out || !g_out) return mm_fail(MM_ERR_INVALID, "NULL array");
  if (c->p.dt > 0 && c->p.dt > stability_guard(c) * (1.0 + 1e-12))
    return mm_fail(MM_ERR_UNSTABLE, "params.dt is above the stability limit");
  cudaSetDevice(c->device);
  const int64_t n = steps_for(t_span, c->dt_limit);
  return fine_impl(c, batch, n, t_span / n, rho_in, g_in, rho_out, g_out, mask_out, c->p.rho_bar, stats,
                   (cudaStream_t)stream);
}

// ------------------------------------------------------------ autotune --

// Time every launch shape F can take for this context on the caller's
// arrays (resident kernel with each cluster size that suits the shape,
// streaming kernel with each lane layout) and keep the fastest for the
// context.  Each candidate runs twice (the first run configures the kernel
// and grows the workspace); the second is timed with events around the
// kernel.
extern "C" mm_status mm_autotune(mm_ctx* c, int32_t batch, int32_t steps, const double* rho_in,
                                 const void* g_in, double* rho_out, void* g_out, mm_tune_result* out,
                                 void* stream) {
  if (!c) return mm_fail(MM_ERR_INVALID, "ctx is NULL");
  if (batch == 0) {  // back to the default choice
    c->tuned = 0;
    c->res_entry = 0;
    if (out) memset(out, 0, sizeof(*out));
    return MM_OK;
  }
  if (batch < 0 || steps < 1) return mm_fail(MM_ERR_INVALID, "batch must be >= 0 and steps >= 1");
  if (!rho_in || !g_in || !rho_out || !g_out) return mm_fail(MM_ERR_INVALID, "NULL array");
  if (g_in == g_out || (const void*)rho_in == (const void*)rho_out)
    return mm_fail(MM_ERR_INVALID, "mm_autotune: outputs must not alias inputs");
  if (c->p.dt > 0 && c->p.dt > stability_guard(c) * (1.0 + 1e-12))
    return mm_fail(MM_ERR_UNSTABLE, "params.dt is above the stability limit");
  cudaSetDevice(c->device);
  const mm_params& p = c->p;
  const bool fp32 = p.precision == MM_FP32G, adapt = p.adapt != 0;
  struct Cand {
    int kernel, C;
    mmk::LaneLayout lay;
    double ms;
  };
  std::vector<Cand> cands;
  if (p.fine_kernel != 1)
    for (int C = 1; C <= 8; C <<= 1)
      if (mmk::fine_resident_smem(p.nx, p.nv, fp32, adapt, p.flux_rule, C)) cands.push_back({2, C, c->lay, 0.0});
  if (p.fine_kernel != 2) {
    const int* vp = fp32 ? kVpt32 : kVpt64;
    for (int q = 0; q < 4; ++q) {
      mmk::LaneLayout lay;
      if (p.fine_vpt && vp[q] != p.fine_vpt) continue;
      if (vpt_offered(p.nv, fp32, vp[q], &lay)) cands.push_back({1, 0, lay, 0.0});
    }
  }
  if (cands.empty()) return mm_fail(MM_ERR_INVALID, "mm_autotune: no launch shape suits this context");
  const int old_tuned = c->tuned, old_kernel = c->tuned_kernel, old_C = c->tuned_cluster;
  const mmk::LaneLayout old_lay = c->tuned_lay;
  const double dt = c->dt_limit;
  size_t best = 0;
  for (size_t q = 0; q < cands.size(); ++q) {
    c->tuned = 1;
    c->tuned_kernel = cands[q].kernel;
    c->tuned_cluster = cands[q].C;
    c->tuned_lay = cands[q].lay;
    mm_fine_stats fs;
    mm_status st = MM_OK;
    for (int rep = 0; rep < 2 && st == MM_OK; ++rep)
      st = fine_impl(c, batch, steps, dt, rho_in, g_in, rho_out, g_out, nullptr, p.rho_bar, &fs,
                     (cudaStream_t)stream);
    if (st != MM_OK) {
      c->tuned = old_tuned;
      c->tuned_kernel = old_kernel;
      c->tuned_cluster = old_C;
      c->tuned_lay = old_lay;
      return st;
    }
    cands[q].ms = fs.elapsed_ms;
    if (cands[q].ms < cands[best].ms) best = q;
  }
  c->tuned = 1;
  c->tuned_kernel = cands[best].kernel;
  c->tuned_cluster = cands[best].C;
  c->tuned_lay = cands[best].lay;
  // Steps per launch of the resident kernel: a batch larger than the GPU
  // holds at once runs in rounds of step chunks, and the chunk count trades
  // the rounds' fill against each chunk's entry and exit (the state's load
  // and store, the field's prefix sum).  That entry cost is measured here,
  // in step-equivalents, from one full wave run for `steps` and for
  // 2 `steps` steps: t(s) = entry + s per_step.
  if (cands[best].kernel == 2) {
    const size_t rs = mmk::fine_resident_smem(p.nx, p.nv, fp32, adapt, p.flux_rule, cands[best].C);
    const int wave = std::min<int>(batch, mmk::resident_capacity(p.nx, p.nv, cands[best].C, rs));
    double t[2] = {0.0, 0.0};
    mm_status st = MM_OK;
    for (int k = 0; k < 2 && st == MM_OK && wave > 0; ++k) {
      mm_fine_stats fs;
      for (int rep = 0; rep < 2 && st == MM_OK; ++rep)
        st = fine_impl(c, wave, (int64_t)steps * (k + 1), dt, rho_in, g_in, rho_out, g_out, nullptr, p.rho_bar, &fs,
                       (cudaStream_t)stream);
      t[k] = fs.elapsed_ms;
    }
    if (st != MM_OK) return st;
    const double per_step = (t[1] - t[0]) / steps;
    c->res_entry = per_step > 0 ? std::min(1000.0, std::max(0.0, (2.0 * t[0] - t[1]) / per_step)) : 0.0;
  } else {
    c->res_entry = 0;
  }
  if (out) {
    memset(out, 0, sizeof(*out));
    out->n_candidates = (int32_t)cands.size();
    out->fine_kernel = cands[best].kernel;
    out->cluster = cands[best].kernel == 2 ? cands[best].C : 1;
    out->vpt = cands[best].lay.vpt;
    out->lanes = cands[best].lay.lanes;
    out->best_ms = cands[best].ms;
    for (size_t q = 0; q < cands.size() && q < 16; ++q) {
      out->cand_kernel[q] = cands[q].kernel;
      out->cand_cluster[q] = cands[q].kernel == 2 ? cands[q].C : 1;
      out->cand_vpt[q] = cands[q].lay.vpt;
      out->cand_ms[q] = cands[q].ms;
    }
    out->res_entry_steps = c->res_entry;
  }
  return MM_OK;
}

// ------------------------------------------------------ coarse and lift --

static mmk::MacroArgs macro_args(const mm_ctx* c, int batch, double t_span, double rho_bar) {
  mmk::MacroArgs a{};
  a.nx = c->p.nx;
  a.nv = c->p.nv;
  a.batch = batch;
  a.dx = c->p.x_len / c->p.nx;
  a.inv_dx = 1.0 / a.dx;
  a.m2 = c->vg.m2;
  a.rho_bar = rho_bar;
  a.eps = c->p.eps;
  a.xiM = c->vg.xiM;
  a.mu3 = c->vg.mu3;
  a.lift_order = c->p.lift_order;
  a.coarse_kind = c->p.coarse_kind;
  a.t_span = t_span;
  int steps = c->p.coarse_steps;
  if (c->p.coarse_kind == 1) {  // explicit S^0: respect its own stability limit
    const double lim = a.dx * a.dx / (2.0 * c->vg.m2) * c->p.cfl_theta;
    steps = std::max<int64_t>(steps, steps_for(t_span, lim));
  }
  a.coarse_steps = steps;
  a.parts = mmk::coarse_parts(a.nx);
  a.vtab = c->d_vtab;
  return a;
}

static double host_mean(const double* rho, int nx, cudaStream_t s, bool* ok) {
  std::vector<double> h(nx);
  *ok = cudaMemcpyAsync(h.data(), rho, nx * sizeof(double), cudaMemcpyDefault, s) == cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess;
  double m = 0.0;
  for (double v : h) m += v;
  return m / nx;
}

extern "C" mm_status mm_coarse(mm_ctx* c, int32_t batch, double t_span, const double* rho_in,
                               double* rho_out, void* stream) {
  if (!c) return mm_fail(MM_ERR_INVALID, "ctx is NULL");
  if (batch < 0 || !(t_span > 0)) return mm_fail(MM_ERR_INVALID, "bad batch or t_span");
  if (batch == 0) return MM_OK;
  if (!rho_in || !rho_out) return mm_fail(MM_ERR_INVALID, "NULL array");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t rbytes = (size_t)batch * c->p.nx * 8;
  void *d_in, *d_out;
  bool s_in, s_out;
  mm_status st;
  if ((st = device_view(c, WS_RHO_IN, rho_in, rbytes, true, s, &d_in, &s_in)) != MM_OK) return st;
  if ((st = device_view(c, WS_RHO_OUT, rho_out, rbytes, false, s, &d_out, &s_out)) != MM_OK) return st;
  double rb = c->p.rho_bar;
  if (isnan(rb)) {
    if (batch != 1) return mm_fail(MM_ERR_INVALID, "rho_bar NaN needs batch == 1 for mm_coarse");
    bool ok;
    rb = host_mean((const double*)d_in, c->p.nx, s, &ok);
    if (!ok) return mm_fail(MM_ERR_CUDA, "mm_coarse: reading rho");
  }
  mmk::MacroArgs a = macro_args(c, batch, t_span, rb);
  void* gws = nullptr;
  const size_t wsb = mmk::macro_ws_bytes(a.nx, batch);
  if (wsb && (st = c->ws.get(WS_MACRO, wsb, s, &gws)) != MM_OK) return st;
  cudaError_t e = mmk::launch_coarse(a, (const double*)d_in, (double*)d_out, (double*)gws, s);
  if (e != cudaSuccess) return mm_cuda_fail(e, "coarse launch");
  if (s_out) {
    CK(cudaMemcpyAsync(rho_out, d_out, rbytes, cudaMemcpyDefault, s), "copy rho_out");
    CK(cudaStreamSynchronize(s), "coarse: synchronise");
  }
  return MM_OK;
}

extern "C" mm_status mm_lift(mm_ctx* c, int32_t batch, const double* rho, void* g_out, void* stream) {
  if (!c) return mm_fail(MM_ERR_INVALID, "ctx is NULL");
  if (batch < 0) return mm_fail(MM_ERR_INVALID, "bad batch");
  if (batch == 0) return MM_OK;
  if (!rho || !g_out) return mm_fail(MM_ERR_INVALID, "NULL array");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const bool fp32 = c->p.precision == MM_FP32G;
  const size_t rbytes = (size_t)batch * c->p.nx * 8;
  const size_t gbytes = (size_t)batch * c->p.nx * c->p.nv * (fp32 ? 4 : 8);
  void *d_in, *d_out;
  bool s_in, s_out;
  mm_status st;
  if ((st = device_view(c, WS_RHO_IN, rho, rbytes, true, s, &d_in, &s_in)) != MM_OK) return st;
  if ((st = device_view(c, WS_G_OUT, g_out, gbytes, false, s, &d_out, &s_out)) != MM_OK) return st;
  double rb = c->p.rho_bar;
  if (isnan(rb)) {
    if (batch != 1) return mm_fail(MM_ERR_INVALID, "rho_bar NaN needs batch == 1 for mm_lift");
    bool ok;
    rb = host_mean((const double*)d_in, c->p.nx, s, &ok);
    if (!ok) return mm_fail(MM_ERR_CUDA, "mm_lift: reading rho");
  }
  mmk::MacroArgs a = macro_args(c, batch, 1.0, rb);
  void* gws = nullptr;
  const size_t wsb = mmk::macro_ws_bytes(a.nx, batch);
  if (wsb && (st = c->ws.get(WS_MACRO, wsb, s, &gws)) != MM_OK) return st;
  cudaError_t e = mmk::launch_lift(a, (const double*)d_in, d_out, fp32, (double*)gws, s);
  if (e != cudaSuccess) return mm_cuda_fail(e, "lift launch");
  if (s_out) {
    CK(cudaMemcpyAsync(g_out, d_out, gbytes, cudaMemcpyDefault, s), "copy g_out");
    CK(cudaStreamSynchronize(s), "lift: synchronise");
  }
  return MM_OK;
}

// ------------------------------------------------------------- parareal --

extern "C" mm_status parareal_run(mm_ctx* c, const mm_parareal_cfg* cfg, const double* rho0, const void* g0,
                                  double* rho_slices_out, mm_parareal_stats* stats, void* stream) {
  if (!c || !cfg) return mm_fail(MM_ERR_INVALID, "NULL argument");
  if (cfg->n_slices < 1 || cfg->max_iter < 0 || !(cfg->t_end > 0))
    return mm_fail(MM_ERR_INVALID, "bad parareal configuration");
  if (cfg->mode != MM_PARAREAL_RHO_LIFT && cfg->mode != MM_PARAREAL_FULL_STATE)
    return mm_fail(MM_ERR_INVALID, "cfg.mode must be MM_PARAREAL_RHO_LIFT or MM_PARAREAL_FULL_STATE");
  const bool full = cfg->mode == MM_PARAREAL_FULL_STATE;
  if (!rho0 || !g0 || !rho_slices_out) return mm_fail(MM_ERR_INVALID, "NULL array");
  if (c->p.dt > 0 && c->p.dt > stability_guard(c) * (1.0 + 1e-12))
    return mm_fail(MM_ERR_UNSTABLE, "params.dt is above the stability limit");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const mm_params& p = c->p;
  const bool fp32 = p.precision == MM_FP32G;
  const int N = cfg->n_slices, nx = p.nx, nv = p.nv;
  const size_t gsz = fp32 ? 4 : 8;
  const size_t rowb = (size_t)nx * 8;
  const double span = cfg->t_end / N;
  const int64_t nf = steps_for(span, c->dt_limit);
  const double dtf = span / nf;

  EventPair ev(true);
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  cudaEventRecord(e0, s);

  mm_status st;
  void *rho, *frho, *gprev, *gb, *errp;
  bool s_out;
  if ((st = device_view(c, WS_PR_RHO, rho_slices_out, rowb * (N + 1), false, s, &rho, &s_out)) != MM_OK)
    return st;
  if ((st = c->ws.get(WS_PR_F, rowb * (N + 1), s, &frho)) != MM_OK) return st;
  if ((st = c->ws.get(WS_PR_G, rowb * (N + 1), s, &gprev)) != MM_OK) return st;
  const size_t G1 = (size_t)nx * nv * gsz;  // bytes of one slice's g
  if ((st = c->ws.get(WS_PR_GB, (size_t)(full ? N + 1 : N) * G1, s, &gb)) != MM_OK) return st;
  if ((st = c->ws.get(WS_PR_ERR, 64, s, &errp)) != MM_OK) return st;
  // full state: the slices' g of the next iterate, the coarse densities
  // before the correction, and the scratch of the lifted differences
  void *gb2 = nullptr, *gold = nullptr, *ldws = nullptr;
  if (full) {
    if ((st = c->ws.get(WS_PR_GB2, (size_t)(N + 1) * G1, s, &gb2)) != MM_OK) return st;
    if ((st = c->ws.get(WS_PR_GOLD, rowb * (N + 1), s, &gold)) != MM_OK) return st;
    if ((st = c->ws.get(WS_PR_LD, mmk::lift_diff_ws_bytes(nx, N), s, &ldws)) != MM_OK) return st;
  }

  // initial slice and rho_bar (mean of the initial density when NaN)
  CK(cudaMemcpyAsync(rho, rho0, rowb, cudaMemcpyDefault, s), "copy rho0");
  double rb = p.rho_bar;
  if (isnan(rb)) {
    bool ok;
    rb = host_mean((const double*)rho, nx, s, &ok);
    if (!ok) return mm_fail(MM_ERR_CUDA, "parareal: reading rho0");
  }
  mmk::MacroArgs ma = macro_args(c, 1, span, rb);
  void* gws = nullptr;
  const size_t wsb = mmk::macro_ws_bytes(nx, std::max(N, 1));
  if (wsb && (st = c->ws.get(WS_MACRO, wsb, s, &gws)) != MM_OK) return st;

  // Overlap of the sequential parts with the fine propagator (density mode,
  // resident kernel in rounds, macro scratch in shared memory so that the
  // two streams share no workspace): the coarse guess and lifting of the
  // slices that the first round does not take run on a second stream during
  // that round, and the correction of the slices whose last chunk has run
  // runs on it during the last round.  The results are those of the
  // sequential order: every dependency is an event.
  const FineChoice fc = fine_choice(c);
  const bool can_overlap = !full && fc.kernel == 2 && wsb == 0;
  auto plan_for = [&](int batch) { return mmk::resident_plan(nx, nv, batch, nf, fc.C, fc.res_smem, c->res_entry); };
  if (can_overlap && !c->side) {
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess) c->side = nullptr;
    for (cudaEvent_t& ev : c->ov)
      if (!ev) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  }
  const bool ov_ok = can_overlap && c->side && c->ov[0] && c->ov[1] && c->ov[2] && c->ov[3];
  cudaStream_t side = c->side;

  int nk = 0;  // kernel launches of this call
  // coarse guess: rho^{n+1,0} = G(rho^{n,0}); with the overlap, slices
  // 1..p-1 (the first round's states) first, the rest on the second stream
  int p_split = 0;  // states of the first round, when the guess is split
  if (ov_ok && N >= 3) {
    const mmk::ResPlan q0 = plan_for(N);
    if (q0.launches() >= 2 && q0.per_round0 >= 2 && q0.per_round0 < N) p_split = q0.per_round0;
  }
  cudaError_t e;
  if (p_split) {
    ++nk;
    e = mmk::launch_coarse_chain(ma, p_split - 1, (double*)rho, (double*)gprev, (double*)gws, s);
    if (e != cudaSuccess) return mm_cuda_fail(e, "coarse guess");
    CK(cudaEventRecord(c->ov[0], s), "overlap event");
    CK(cudaStreamWaitEvent(side, c->ov[0], 0), "overlap wait");
    ++nk;
    e = mmk::launch_coarse_chain(ma, N - p_split + 1, (double*)rho + (size_t)(p_split - 1) * nx,
                                 (double*)gprev + (size_t)(p_split - 1) * nx, (double*)gws, side, false);
    if (e != cudaSuccess) return mm_cuda_fail(e, "coarse guess");
    mmk::MacroArgs la = macro_args(c, N - p_split, span, rb);
    ++nk;
    e = mmk::launch_lift(la, (const double*)rho + (size_t)p_split * nx, (char*)gb + (size_t)p_split * G1, fp32,
                         (double*)gws, side);
    if (e != cudaSuccess) return mm_cuda_fail(e, "lift");
    CK(cudaEventRecord(c->ov[1], side), "overlap event");
  } else {
    ++nk;
    e = mmk::launch_coarse_chain(ma, N, (double*)rho, (double*)gprev, (double*)gws, s);
    if (e != cudaSuccess) return mm_cuda_fail(e, "coarse guess");
  }

  int it = 0;
  int64_t kin_total = 0;
  double fine_ms = 0.0;
  int fine_launches = 0;
  EventPair fev(stats != nullptr);
  FineDefer fd;
  fd.e0 = fev.a;
  fd.e1 = fev.b;
  const int K = std::min(cfg->max_iter, N);
  for (int k = 0; k < K; ++k) {
    const int batch = N - k;
    // inputs of the fine propagations: (rho^{n,k}, g^{n,k}), n = k..N-1.
    // Density mode: g relifted from the density into gb[0..batch) (slice 0
    // from g0).  Full state: the slices' own g, kept at gb[n] (lifted once
    // from the coarse guess).
    mmk::ResHooks hooks{};
    bool use_hooks = false;
    if (k == 0) {
      CK(cudaMemcpyAsync(gb, g0, (size_t)nx * nv * gsz, cudaMemcpyDefault, s), "copy g0");
      const int n_lift = p_split ? p_split - 1 : N - 1;  // slices 1..n_lift here
      if (n_lift > 0) {
        mmk::MacroArgs la = macro_args(c, n_lift, span, rb);
        ++nk;
        e = mmk::launch_lift(la, (const double*)rho + nx, (char*)gb + G1, fp32, (double*)gws, s);
      }
      if (p_split) {  // the second round needs the rest of the guess and its lifting
        hooks.before[1] = c->ov[1];
        use_hooks = true;
      }
    } else if (!full) {
      mmk::MacroArgs la = macro_args(c, batch, span, rb);
      ++nk;
      e = mmk::launch_lift(la, (const double*)rho + (size_t)k * nx, gb, fp32, (double*)gws, s);
    }
    if (e != cudaSuccess) return mm_cuda_fail(e, "lift");
    void* g_in = full ? (void*)((char*)gb + (size_t)k * G1) : gb;
    void* g_out = full ? (void*)((char*)gb2 + (size_t)(k + 1) * G1) : gb;  // full: F_g(U^{n,k}) at n+1
    // correction split: the states final before the last launch (a prefix,
    // the items being chunk-major) are corrected during it
    int m_split = 0;
    if (ov_ok) {
      const mmk::ResPlan q = plan_for(batch);
      const int j = q.launches() - 2;
      if (j >= 0 && j < mmk::ResHooks::kMax) {
        while (m_split < batch && q.final_launch(m_split) <= j) ++m_split;
        if (m_split >= batch) m_split = 0;
        if (m_split) {
          hooks.after[j] = c->ov[2];
          use_hooks = true;
        }
      }
    }
    st = fine_impl(c, batch, nf, dtf, (const double*)rho + (size_t)k * nx, g_in,
                   (double*)frho + (size_t)(k + 1) * nx, g_out, nullptr, rb, nullptr, s,
                   use_hooks ? &hooks : nullptr, &fd);
    if (st != MM_OK) return st;
    // sequential correction on the device (the coarse values before it are
    // kept for the full-state g correction)
    if (full) CK(cudaMemcpyAsync(gold, gprev, rowb * (N + 1), cudaMemcpyDeviceToDevice, s), "save G");
    mmk::CorrectArgs ca{};
    ca.m = ma;
    ca.n_slices = N;
    ca.k = k;
    ca.rho = (double*)rho;
    ca.frho = (const double*)frho;
    ca.gprev = (double*)gprev;
    ca.err = (double*)errp;
    if (m_split) {  // slices k..k+m-1 on the second stream, then the rest
      mmk::CorrectArgs c1 = ca;
      c1.n_slices = k + m_split;
      CK(cudaStreamWaitEvent(side, c->ov[2], 0), "overlap wait");
      ++nk;
      e = mmk::launch_correct(c1, (double*)gws, side, false);
      if (e != cudaSuccess) return mm_cuda_fail(e, "correction");
      CK(cudaEventRecord(c->ov[3], side), "overlap event");
      CK(cudaStreamWaitEvent(s, c->ov[3], 0), "overlap join");
      ca.k = k + m_split;
      ca.err = (double*)errp + 1;
    }
    ++nk;
    e = mmk::launch_correct(ca, (double*)gws, s);
    if (e != cudaSuccess) return mm_cuda_fail(e, "correction");
    if (full) {  // g^{n+1,k+1} = F_g(U^{n,k}) + (L G rho^{n,k+1} - L G rho^{n,k}), n = k..N-1
      mmk::MacroArgs la = macro_args(c, batch, span, rb);
      ++nk;
      e = mmk::launch_lift_diff(la, (const double*)gprev + (size_t)(k + 1) * nx,
                                (const double*)gold + (size_t)(k + 1) * nx, (char*)gb2 + (size_t)(k + 1) * G1,
                                fp32, (double*)ldws, s);
      if (e != cudaSuccess) return mm_cuda_fail(e, "full-state correction");
      std::swap(gb, gb2);
    }
    double errs[2] = {0.0, 0.0};
    int hs[6] = {0};
    CK(cudaMemcpyAsync(errs, errp, m_split ? 16 : 8, cudaMemcpyDeviceToHost, s), "read error");
    CK(cudaMemcpyAsync(hs, fd.status, 24, cudaMemcpyDeviceToHost, s), "read fine status");
    CK(cudaStreamSynchronize(s), "parareal: synchronise");
    if (hs[0] != 0) return mm_fail((mm_status)hs[0], "fine: non-finite density");
    if (stats) {
      float ms = 0;
      cudaEventElapsedTime(&ms, fd.e0, fd.e1);
      unsigned long long kc;
      memcpy(&kc, (char*)hs + 16, 8);
      kin_total += (int64_t)kc;
      fine_ms += ms;
      fine_launches += fd.launches;
    }
    nk += fd.launches;
    const double err = std::max(errs[0], errs[1]);
    if (stats && k < 64) stats->err[k] = err;
    ++it;
    if (err < cfg->tol) break;
  }
  cudaEventRecord(e1, s);
  if (s_out) CK(cudaMemcpyAsync(rho_slices_out, rho, rowb * (N + 1), cudaMemcpyDefault, s), "copy slices");
  CK(cudaStreamSynchronize(s), "parareal: final synchronise");
  if (stats) {
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    stats->iterations = it;
    stats->fine_steps = nf;
    stats->kinetic_updates = kin_total;
    stats->elapsed_ms = ms;
    stats->fine_ms = fine_ms;
    stats->fine_launches = fine_launches;
    // mass of every slice, summed on the device (N + 1 doubles come back)
    void* sums;
    if ((st = c->ws.get(WS_PR_SUM, (size_t)(N + 1) * 8, s, &sums)) != MM_OK) return st;
    ++nk;
    e = mmk::launch_row_sums((const double*)rho, N + 1, nx, (double*)sums, s);
    if (e != cudaSuccess) return mm_cuda_fail(e, "mass sums");
    std::vector<double> m((size_t)N + 1);
    CK(cudaMemcpyAsync(m.data(), sums, (size_t)(N + 1) * 8, cudaMemcpyDeviceToHost, s), "read mass sums");
    CK(cudaStreamSynchronize(s), "parareal: mass sums");
    double drift = 0;
    for (int n = 1; n <= N; ++n) drift = std::max(drift, fabs(m[n] - m[0]) / fabs(m[0]));
    stats->mass_drift = drift;
    stats->kernel_launches = nk;
  }
  return MM_OK;
}

extern "C" mm_status mm_set_chunk_entry(mm_ctx* c, double entry_steps) {
  if (!c) return mm_fail(MM_ERR_INVALID, "ctx is NULL");
  if (!(entry_steps >= 0.0 && entry_steps <= 1000.0)) return mm_fail(MM_ERR_INVALID, "entry_steps outside [0, 1000]");
  c->res_entry = entry_steps;
  return MM_OK;
}

// --------------------------------------------- fine plan without buffers --

// Kernel arguments of F for one call, with every buffer pointer left unset
// (used by the entry point that takes its scratch from static device
// memory instead of the workspace).
// ------------------------------------------- parareal building blocks --

// Algorithm 1's sequential parts as separate calls, for drivers that run
// the fine propagations of one iteration on several devices (each device
// its block of slices, the results gathered, the sequential part redone on
// every device).  Device arrays only.
static mm_status parareal_rb(mm_ctx* c, const double* rho_slices, cudaStream_t s, double* rb) {
  *rb = c->p.rho_bar;
  if (isnan(*rb)) {
    bool ok;
    *rb = host_mean(rho_slices, c->p.nx, s, &ok);
    if (!ok) return mm_fail(MM_ERR_CUDA, "parareal: reading slice 0");
  }
  return MM_OK;
}

extern "C" mm_status mm_coarse_guess(mm_ctx* c, int32_t n_slices, double t_span, double* rho_slices,
                                     double* g_prev, void* stream) {
  if (!c) return mm_fail(MM_ERR_INVALID, "ctx is NULL");
  if (n_slices < 1 || !(t_span > 0)) return mm_fail(MM_ERR_INVALID, "n_slices must be >= 1 and t_span > 0");
  if (!rho_slices || !g_prev) return mm_fail(MM_ERR_INVALID, "NULL array");
  if (!is_device_ptr(rho_slices) || !is_device_ptr(g_prev))
    return mm_fail(MM_ERR_INVALID, "mm_coarse_guess takes device arrays");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  double rb;
  mm_status st = parareal_rb(c, rho_slices, s, &rb);
  if (st != MM_OK) return st;
  mmk::MacroArgs ma = macro_args(c, 1, t_span, rb);
  void* gws = nullptr;
  const size_t wsb = mmk::macro_ws_bytes(c->p.nx, std::max((int)n_slices, 1));
  if (wsb && (st = c->ws.get(WS_MACRO, wsb, s, &gws)) != MM_OK) return st;
  const cudaError_t e = mmk::launch_coarse_chain(ma, n_slices, rho_slices, g_prev, (double*)gws, s);
  if (e != cudaSuccess) return mm_cuda_fail(e, "coarse guess");
  return MM_OK;
}

extern "C" mm_status mm_parareal_correct(mm_ctx* c, int32_t n_slices, int32_t k, double t_span,
                                         double* rho_slices, const double* f_rho, double* g_prev,
                                         double* err, void* stream) {
  if (!c) return mm_fail(MM_ERR_INVALID, "ctx is NULL");
  if (n_slices < 1 || k < 0 || k >= n_slices || !(t_span > 0))
    return mm_fail(MM_ERR_INVALID, "need n_slices >= 1, 0 <= k < n_slices and t_span > 0");
  if (!rho_slices || !f_rho || !g_prev || !err) return mm_fail(MM_ERR_INVALID, "NULL array");
  if (!is_device_ptr(rho_slices) || !is_device_ptr(f_rho) || !is_device_ptr(g_prev) || !is_device_ptr(err))
    return mm_fail(MM_ERR_INVALID, "mm_parareal_correct takes device arrays");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  double rb;
  mm_status st = parareal_rb(c, rho_slices, s, &rb);
  if (st != MM_OK) return st;
  void* gws = nullptr;
  const size_t wsb = mmk::macro_ws_bytes(c->p.nx, std::max((int)n_slices, 1));
  if (wsb && (st = c->ws.get(WS_MACRO, wsb, s, &gws)) != MM_OK) return st;
  mmk::CorrectArgs ca{};
  ca.m = macro_args(c, 1, t_span, rb);
  ca.n_slices = n_slices;
  ca.k = k;
  ca.rho = rho_slices;
  ca.frho = f_rho;
  ca.gprev = g_prev;
  ca.err = err;
  const cudaError_t e = mmk::launch_correct(ca, (double*)gws, s);
  if (e != cudaSuccess) return mm_cuda_fail(e, "correction");
  return MM_OK;
}

mm_status mmk::fine_plan(mm_ctx* c, int32_t batch, double t_span, FinePlan* out, bool check_dt) {
  if (!c) return mm_fail(MM_ERR_INVALID, "ctx is NULL");
  if (batch < 0) return mm_fail(MM_ERR_INVALID, "batch must be >= 0");
  if (!(t_span > 0)) return mm_fail(MM_ERR_INVALID, "t_span must be > 0");
  if (check_dt && c->p.dt > 0 && c->p.dt > stability_guard(c) * (1.0 + 1e-12))
    return mm_fail(MM_ERR_UNSTABLE, "params.dt is above the stability limit");
  const mm_params& p = c->p;
  const int64_t n = steps_for(t_span, c->dt_limit);
  const double dt = t_span / n;
  const FineChoice fc = fine_choice(c);
  FinePlan f{};
  f.device = c->device;
  f.fp32 = p.precision == MM_FP32G;
  f.vpt = fc.lay.vpt;
  f.kernel = fc.kernel;
  f.res_C = fc.kernel == 2 ? fc.C : 0;
  f.res_smem = fc.kernel == 2 ? fc.res_smem : 0;
  f.n_steps = n;
  f.g_bytes = (size_t)batch * p.nx * p.nv * (f.fp32 ? 4 : 8);
  f.rho_bytes = (size_t)batch * p.nx * 8;
  const bool adapt = p.adapt != 0;
  f.col_bytes = mmk::fine_column_bytes(p.nx, p.nv, fc.lay.lanes, f.fp32, adapt, false);
  f.col_in_smem = f.col_bytes == 0;
  f.smem = mmk::fine_smem_bytes(p.nx, p.nv, fc.lay.lanes, f.fp32, adapt, false);
  FineArgs& a = f.args;
  a.nx = p.nx;
  a.nv = p.nv;
  a.batch = batch;
  a.n_steps = n;
  a.lanes = fc.lay.lanes;
  a.nh = fc.lay.nh;
  a.nhp = fc.lay.nhp;
  a.dt = dt;
  a.dx = p.x_len / p.nx;
  a.inv_dx = 1.0 / a.dx;
  a.inv_dv = 1.0 / c->vg.dv;
  a.eps = p.eps;
  a.inv_eps = 1.0 / p.eps;
  a.a = exp(-dt / (p.eps * p.eps));
  a.b = p.eps * (1.0 - a.a);
  a.m2 = c->vg.m2;
  a.dt_dx = dt / a.dx;
  a.rho_bar = p.rho_bar;
  a.adapt = p.adapt;
  a.r_scale = p.r_scale;
  a.flux_rule = p.flux_rule;
  a.thr_g = p.thr_g;
  a.thr_R = p.thr_R;
  a.r_fac = p.r_scale ? p.eps * p.eps : 1.0;
  a.vtab = c->d_vtab;
  a.vtab_f = c->d_vtab_f;
  a.xiM = c->vg.xiM;
  a.mu3 = c->vg.mu3;
  a.lift_order = c->p.lift_order;
  a.res_entry_steps = c->res_entry;
  a.col_in_smem = f.col_in_smem ? 1 : 0;
  a.col_ws_stride = f.col_in_smem ? 0 : f.col_bytes;
  *out = f;
  return MM_OK;
}

// ------------------------------------------- context access for batches --

const mm_params& mmk::ctx_params(const mm_ctx* c) { return c->p; }
double mmk::solve_iteration_cost(const mm_params& p, const mm_parareal_cfg& cfg) {
  if (p.nv < 4 || p.nx < 1 || cfg.n_slices < 1 || !(cfg.t_end > 0)) return 0.0;
  mm_params q = p;
  if (q.cfl_theta == 0) q.cfl_theta = 0.9;
  const mmk::VelocityGrid vg = build_velocity_grid(p.nv, p.v_max);
  const double lim = q.dt > 0 ? q.dt : q.cfl_theta * stability_limit(q, vg.m2);
  const double steps = (double)steps_for(cfg.t_end / cfg.n_slices, lim);
  return (double)p.nx * p.nv * cfg.n_slices * steps;
}
int mmk::ctx_device(const mm_ctx* c) { return c->device; }
int64_t mmk::ctx_fine_steps(const mm_ctx* c, double span) { return steps_for(span, c->dt_limit); }
mmk::MacroArgs mmk::ctx_macro_args(const mm_ctx* c, double span, double rho_bar) {
  return macro_args(c, 1, span, rho_bar);
}
double mmk::ctx_mean(const double* rho, int nx) {
  double m = 0.0;
  for (int i = 0; i < nx; ++i) m += rho[i];
  return m / nx;
}

mmk::FineArgs mmk::ctx_fine_args(const mm_ctx* c, int64_t n, double dt, double rho_bar) {
  const mm_params& p = c->p;
  FineArgs a{};
  a.nx = p.nx;
  a.nv = p.nv;
  a.batch = 1;
  a.n_steps = n;
  a.lanes = c->lay.lanes;
  a.nh = c->lay.nh;
  a.nhp = c->lay.nhp;
  a.dt = dt;
  a.dx = p.x_len / p.nx;
  a.inv_dx = 1.0 / a.dx;
  a.inv_dv = 1.0 / c->vg.dv;
  a.eps = p.eps;
  a.inv_eps = 1.0 / p.eps;
  a.a = exp(-dt / (p.eps * p.eps));
  a.b = p.eps * (1.0 - a.a);
  a.m2 = c->vg.m2;
  a.dt_dx = dt / a.dx;
  a.rho_bar = rho_bar;
  a.adapt = p.adapt;
  a.r_scale = p.r_scale;
  a.flux_rule = p.flux_rule;
  a.thr_g = p.thr_g;
  a.thr_R = p.thr_R;
  a.r_fac = p.r_scale ? p.eps * p.eps : 1.0;
  a.vtab = c->d_vtab;
  a.vtab_f = c->d_vtab_f;
  a.xiM = c->vg.xiM;
  a.mu3 = c->vg.mu3;
  a.lift_order = c->p.lift_order;
  fine_args_floats(a);
  return a;
}

// The lane layout a work list runs with: 8 nodes per lane in FP32, 4 in FP64
// (the persistent kernel is compiled for those only).
bool mmk::ctx_list_layout(const mm_ctx* c, int* lanes) {
  const bool fp32 = c->p.precision == MM_FP32G;
  *lanes = c->lay.lanes;
  return c->lay.vpt == (fp32 ? 8 : 4);
}
