// Internal declarations shared by the host API and the kernels of libmm.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mm.h"

namespace mmk {

constexpr int kFineThreads = 512;   // threads of one fine CTA (one state)
constexpr int kResThreads = 256;    // threads of one CTA of the resident kernel
constexpr int kVTabFields = 6;      // per velocity node: |v|/dx, M, v M, w v, w, v

// Velocity constants of one context, built on the host in double.
struct VelocityGrid {
  int nv = 0;
  double dv = 0, m2 = 0, xiM = 0, mu3 = 0;  // m2 = <v^2 M>, xiM = <v M>, mu3 = <v^3 M>
  std::vector<double> v, w, M;
};

// Lane layout of the fine sweep: each interface column is handled by a
// group of `lanes` consecutive lanes (a power of two <= 32); lane l of the
// negative half owns nodes [l*vpt, (l+1)*vpt), lane nhp+l of the positive
// half owns nodes [nv/2 + l*vpt, ...); lanes with l >= nh are idle.
struct LaneLayout {
  int vpt = 0, lanes = 0, nh = 0, nhp = 0;
};

// Arguments of the fine kernel (plain data; device pointers).
struct FineArgs {
  int nx, nv, batch;
  int64_t n_steps;
  int lanes, nh, nhp;
  double dt, dx, inv_dx, inv_dv, eps, inv_eps, a, b, m2, dt_dx;
  double rho_bar;       // NaN: mean of each state's density
  int adapt, r_scale, flux_rule;
  double thr_g, thr_R, r_fac;
  const double* rho_in;
  double* rho_out;
  const void* g_in;
  void* g_buf0;         // step buffers: step s writes buf[(n_steps-1-s)&1]
  void* g_buf1;         //   so the last step writes buf0 (= g_out)
  uint8_t* mask_out;
  const double* vtab;   // [kVTabFields][nv] in double
  const float* vtab_f;  // same in float
  void* col_ws;         // per-state column arrays when they do not fit smem
  size_t col_ws_stride; // bytes per state in col_ws
  int col_in_smem;      // 1: column arrays in shared memory
  unsigned long long* kin_count;  // kinetic cell-updates (summed)
  int* status;          // device status word (mm_status)
  // float copies of the scalars, rounded once on the host so that no FP64
  // instruction is needed (or re-issued) inside the FP32 kernels' step loop
  float fa, fb, f_dx, f_inv_dx, f_inv_dv, f_kflux, f_fflux, f_inv_nx;
  float f_dx_lo, f_inv_nx_lo;  // low parts of dx and 1/nx as float-float
  // adaptation criteria of the FP32 path: 1/(60 dx) as float-float (first
  // derivative stencil of Table 1 with integer weights), 1/(180 dx^2),
  // 1/(8 dx^3), thr_g^2, thr_R, r_fac
  float f_k1, f_k1_lo, f_k2, f_k3, f_thr_g2, f_thr_R, f_rfac;
  double xiM;                  // <xi M> of the discrete Maxwellian (lifting)
  double mu3;                  // <xi^3 M> (lifting of order three)
  int lift_order;              // order L of the lifting (Def. 1), 1..3
  // resident kernel: first work item of this launch, and whether the
  // launch's first chunk of each state reads the input (set by
  // launch_fine_resident)
  int res_item0, res_from_input;
  int res_state0;               // res_item0 mod batch
  // resident kernel: cost of a chunk's entry and exit in step-equivalents,
  // as measured by mm_autotune (0: the built-in estimate)
  double res_entry_steps;
};

// Work list of fine propagations across solves (persistent kernel).
struct FineListSolve {
  FineArgs a;          // the solve's constants (shape, steps, dt, ...)
  const double* rho;   // [N+1][nx] slice densities rho^{n,k} (input of slice n)
  double* frho;        // [N+1][nx] F(rho^{n,k}) written at n+1
  const void* g0;      // slice 0's perturbation (context precision) or null
};
struct FineListItem {
  int solve, slice;
};
struct FineList {
  const FineListSolve* solves;
  const FineListItem* items;
  int n_items, grid;
  int* next;            // work counter, zero at launch
  unsigned char* ws;    // per CTA: two step buffers of ws_g bytes (+ ws_col)
  size_t ws_g, ws_col;
};
// Launch the persistent list kernel: FP32 (8 nodes per lane) or FP64 (4);
// every solve of the list must share precision and adaptation.
cudaError_t launch_fine_list(const FineList& L, bool fp32, bool adapt, size_t smem, cudaStream_t s);

// Fill the float copies of a FineArgs from its double fields.
inline void fine_args_floats(FineArgs& a) {
  a.fa = (float)a.a;
  a.fb = (float)a.b;
  a.f_dx = (float)a.dx;
  a.f_dx_lo = (float)(a.dx - (double)a.f_dx);
  a.f_inv_dx = (float)a.inv_dx;
  a.f_inv_dv = (float)a.inv_dv;
  a.f_kflux = (float)(a.dt_dx * a.inv_eps);
  a.f_fflux = (float)(-a.dt_dx * a.m2);
  a.f_inv_nx = (float)(1.0 / a.nx);
  a.f_inv_nx_lo = (float)(1.0 / a.nx - (double)a.f_inv_nx);
  const double k1 = a.inv_dx / 60.0;
  a.f_k1 = (float)k1;
  a.f_k1_lo = (float)(k1 - (double)a.f_k1);
  a.f_k2 = (float)(a.inv_dx * a.inv_dx / 180.0);
  a.f_k3 = (float)(a.inv_dx * a.inv_dx * a.inv_dx / 8.0);
  a.f_thr_g2 = (float)(a.thr_g * a.thr_g);
  a.f_thr_R = (float)a.thr_R;
  a.f_rfac = (float)a.r_fac;
}

// Column arrays of one state: the bytes that go to global memory (0 when
// all of them fit shared memory) and the kernel's dynamic shared memory,
// for the fine kernel (list = false) or the work-list kernel (list = true).
size_t fine_column_bytes(int nx, int nv, int lanes, bool fp32, bool adapt, bool list);
size_t fine_smem_bytes(int nx, int nv, int lanes, bool fp32, bool adapt, bool list);

// Launch the fine kernel for a batch (one CTA per state).
cudaError_t launch_fine(const FineArgs& a, int vpt, bool fp32, size_t smem,
                        cudaStream_t s);

// Resident variant of F (g kept in shared memory across the whole launch,
// one thread-block cluster per state).  fine_resident_cluster returns the
// cluster size (0: shape not supported) and the dynamic shared memory.
int fine_resident_cluster(int nx, int nv, bool fp32, bool adapt, int flux_rule, size_t* smem);
size_t fine_resident_smem(int nx, int nv, bool fp32, bool adapt, int flux_rule, int C);
// Launch plan of the resident kernel for one call: a batch larger than the
// GPU holds at once runs as batch x chunks items of L steps in rounds
// (launches0 launches), then the r steps left over (launches1 launches).
struct ResPlan {
  int batch, chunks;
  int64_t L, r;
  int per_round0, per_round1, launches0, launches1;
  int launches() const { return launches0 + launches1; }
  int final_launch(int state) const;  // the launch after which the state is final
};
// entry_steps: a chunk's entry and exit cost in step-equivalents (0: the
// built-in estimate)
ResPlan resident_plan(int nx, int nv, int batch, int64_t n_steps, int C, size_t smem, double entry_steps = 0.0);
// Clusters of the resident kernel the GPU holds at once for a shape.
int resident_capacity(int nx, int nv, int C, size_t smem);
// Events around the launches of one call (null entries are skipped): the
// stream waits for before[i] ahead of launch i and records after[i] behind it.
struct ResHooks {
  static constexpr int kMax = 64;
  cudaEvent_t before[kMax];
  cudaEvent_t after[kMax];
};
// *launches (nullable) receives the kernel launches made.
cudaError_t launch_fine_resident(const FineArgs& a, int C, size_t smem, cudaStream_t s, int* launches = nullptr,
                                 const ResHooks* hooks = nullptr);

// Arguments of the macroscopic kernels (coarse step, lift, correction).
struct MacroArgs {
  int nx, nv, batch;
  double dx, inv_dx, m2, rho_bar, eps, xiM, mu3;
  int lift_order;       // order L of the lifting (Def. 1), 1..3
  int coarse_kind, coarse_steps;
  int parts;            // chunks of the partitioned tridiagonal solve
  double t_span;
  const double* vtab;   // [kVTabFields][nv]
};

// Global scratch (doubles) the macroscopic kernels need for `grid` CTAs when
// their arrays do not fit shared memory (0 when they fit).
size_t macro_ws_bytes(int nx, int grid);
int coarse_parts(int nx);
cudaError_t launch_coarse(const MacroArgs& a, const double* rho_in, double* rho_out, double* gws,
                          cudaStream_t s);
cudaError_t launch_lift(const MacroArgs& a, const double* rho, void* g_out, bool fp32, double* gws,
                        cudaStream_t s);
// Full-state parareal: g[b] += L rho_new[b] - L rho_old[b] for a.batch
// densities; ws holds lift_diff_ws_bytes(nx, batch) bytes.
size_t lift_diff_ws_bytes(int nx, int batch);
cudaError_t launch_lift_diff(const MacroArgs& a, const double* rho_new, const double* rho_old, void* g, bool fp32,
                             double* ws, cudaStream_t s);

// Parareal on the device: the sequential correction sweep over slices
// n = k..N-1 (one CTA per solve), and the successive-error reduction.
struct CorrectArgs {
  MacroArgs m;
  int n_slices, k;
  double* rho;          // [N+1][nx]  rho^{n,k} in, rho^{n,k+1} out
  const double* frho;   // [N+1][nx]  F(rho^{n,k}) at index n+1
  double* gprev;        // [N+1][nx]  G(rho^{n,k}) at index n+1 (updated)
  double* err;          // one double: max_n,i |rho^{n,k+1} - rho^{n,k}|
  double* work;         // [nx] scratch per solve
};
// cluster: allow the variant that spreads one solve's implicit step over a
// thread-block cluster (mm_coarse_cluster.cu) where the shape suits it; the
// launches that run beside the fine kernel's rounds keep the one-CTA
// kernel, which fits on an SM the rounds leave free.
cudaError_t launch_correct(const CorrectArgs& a, double* gws, cudaStream_t s, bool cluster = true);
cudaError_t launch_coarse_chain(const MacroArgs& a, int n_slices, double* rho, double* gprev,
                                double* gws, cudaStream_t s, bool cluster = true);
bool coarse_cluster_ok(const MacroArgs& a);
cudaError_t launch_coarse_chain_cluster(const MacroArgs& a, int n_slices, double* rho, double* gprev,
                                        cudaStream_t s);
cudaError_t launch_correct_cluster(const CorrectArgs& c, cudaStream_t s);
// The same for n solves of one grid size nx (coarse_cluster_ok), one cluster
// each; `list` in device memory.
cudaError_t launch_coarse_chain_cluster_list(const CorrectArgs* list, int n, int nx, cudaStream_t s);
cudaError_t launch_correct_cluster_list(const CorrectArgs* list, int n, int nx, cudaStream_t s);
// out[r] = sum of row r of x ([rows][nx]): the slices' mass, which the
// parareal driver reports as its mass drift.
cudaError_t launch_row_sums(const double* x, int rows, int nx, double* out, cudaStream_t s);
// Many solves, one CTA each; `list` in device memory; scratch for nx_max.
size_t macro_list_ws_bytes(int nx_max, int grid);
cudaError_t launch_correct_list(const CorrectArgs* list, int n, int nx_max, double* gws, cudaStream_t s);
cudaError_t launch_coarse_chain_list(const CorrectArgs* list, int n, int nx_max, double* gws, cudaStream_t s);

// Everything the fine kernel needs for one call except its buffers: the
// arguments (pointers unset), the template choice and the byte counts.
// The kernel and launch shape are those mm_fine_propagate would use for the
// context (its tuned choice, else the default rule).
struct FinePlan {
  FineArgs args;
  int device, vpt;
  bool fp32, col_in_smem;
  int64_t n_steps;
  size_t g_bytes, rho_bytes, col_bytes, smem;
  int kernel;          // 1 streaming, 2 resident
  int res_C;           // resident: CTAs per state
  size_t res_smem;     // resident: dynamic shared memory
};
// check_dt: refuse a params.dt above the stability rule (MM_ERR_UNSTABLE).
mm_status fine_plan(mm_ctx* c, int32_t batch, double t_span, FinePlan* out, bool check_dt = true);
// Load the kernel instances a plan launches (under lazy module loading a
// first launch would otherwise load them, which can allocate device memory).
cudaError_t fine_preload(const FinePlan& f);
cudaError_t fine_stream_preload(const FineArgs& a, int vpt, bool fp32);
// Set-up of mm_fine_propagate_noalloc for a context's device, done by
// mm_create: the device address of the fixed scratch array, and the
// kernels of the context's launch choice loaded.
mm_status noalloc_setup(mm_ctx* c);

// Free a context without a device-wide synchronisation (stream-ordered on s).
void ctx_release(mm_ctx* c, cudaStream_t s);

// Context access for the batch engine (mm_batch.cpp).
const mm_params& ctx_params(const mm_ctx* c);
int ctx_device(const mm_ctx* c);
int64_t ctx_fine_steps(const mm_ctx* c, double span);
MacroArgs ctx_macro_args(const mm_ctx* c, double span, double rho_bar);
FineArgs ctx_fine_args(const mm_ctx* c, int64_t n, double dt, double rho_bar);  // pointers unset
bool ctx_list_layout(const mm_ctx* c, int* lanes);
// Fine cell-updates of one parareal iteration of a solve (every slice, the
// whole window of steps, all cells), from the step rule on the host: the
// serving scheduler's cost estimate.
double solve_iteration_cost(const mm_params& p, const mm_parareal_cfg& c);
// Cap on the CTAs of a batch's work-list launch (0: one per SM); lets two
// batches share the GPU on disjoint SMs.
void batch_set_max_ctas(mm_batch* b, int n);
// Grid from which a batch runs a solve's coarse guess and correction over a
// thread-block cluster instead of one CTA (4096 unless set).
void batch_set_cluster_min_nx(mm_batch* b, int nx);
// The server's lanes share the GPU: clusters only for the largest grids.
constexpr int kServeClusterMinNx = 16384;
double ctx_mean(const double* rho, int nx);

}  // namespace mmk

// Thread-local error message helpers (mm_api.cpp).
mm_status mm_fail(mm_status st, const std::string& msg);
mm_status mm_cuda_fail(cudaError_t e, const char* what);
