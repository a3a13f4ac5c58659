// The linearly implicit coarse step (S^0, Sec. 2.3) of one density spread
// over a thread-block cluster: the coarse guess and the sequential
// correction of Algorithm 1 (Sec. 3.3) for a single solve.
//
// Why this shape.  The step is a cyclic tridiagonal solve in double, and
// GB300's FP64 pipe takes 64 cycles to issue one warp-wide FP64
// instruction on its SM sub-partition, however many lanes are active (two
// lanes per clock per SM; one lane active costs the same as 32).  So the
// time of a step is the number of dependent FP64 instructions on the
// busiest warp, plus the cluster barriers; lanes are free.  Hence:
//   - one row per thread, nb = nx / kCC rows per CTA, nb / 32 warps per
//     CTA (one per sub-partition at Nx = 1024);
//   - each warp eliminates its 31 interior rows by parallel cyclic
//     reduction in registers (shuffles, no barrier), with three right-hand
//     sides: the data and the couplings to its two bounding separators
//     (the previous warp's last row and its own last row);
//   - the nx / 32 warp separators form a cyclic tridiagonal system that
//     every warp assembles from the records of all warps (one exchange
//     through distributed shared memory) and solves redundantly by
//     parallel cyclic reduction in registers;
//   - every row is then rebuilt from its two separator values.
// Two cluster barriers per step, against one per reduction level when the
// reduction itself is distributed over the cluster; about 11 us per step at
// Nx = 1024 against 16 us for that layout.
//
// Per step:
//   1. the Poisson law of S^MM for the frozen field: a warp scan of the
//      density deviations, the warps' totals through shared memory, the
//      CTAs' totals through distributed shared memory;
//   2. the coefficients of (I - m2 dt L_E) x = rho;
//   3. the warp-local reduction;
//   4. the separator records, one cluster barrier, the separators' system;
//   5. the rows rebuilt.
#include <cooperative_groups.h>

#include "mm_internal.h"

namespace cg = cooperative_groups;

namespace mmk {

namespace {

constexpr int kCC = 8;  // CTAs per cluster
constexpr unsigned kFull = 0xffffffffu;

template <class P>
__device__ __forceinline__ P* on_rank(P* p, int rank) {
  return cg::this_cluster().map_shared_rank(p, rank);
}

// Shared memory of one CTA (doubles).
struct CMap {
  double* E;    // [nb] field at the CTA's rows
  double* rec;  // [nw][8] separator record of each warp
  double* ex;   // [kCC][2] the CTAs' Poisson totals (pushed by every CTA)
  double* wt;   // [2][8] the warps' Poisson totals
  double* em;   // [kCC] the CTAs' maximum corrections (rank 0's copy)
};

__host__ __device__ inline size_t cmap_doubles(int nb) { return (size_t)nb + 8 * (nb / 32) + 2 * kCC + 16 + kCC; }

__device__ CMap carve_cmap(double* base, int nb) {
  CMap m;
  m.E = base;
  m.rec = m.E + nb;
  m.ex = m.rec + 8 * (nb / 32);
  m.wt = m.ex + 2 * kCC;
  m.em = m.wt + 16;
  return m;
}

// Per-thread constants of a chain: the row's weight nx - g in the mean of
// the Poisson prefix sums, and 1 / nx.
struct RowConst {
  double wgt, inv_nx;
};

// One linearly implicit S^0 step of the cluster's density; w is this
// thread's row of rho, the result its row of (I - m2 dt L_E)^{-1} rho with
// E frozen from rho.
__device__ double implicit_step_cluster(const CMap& M, const MacroArgs& a, double dt, int nb, int r, double w,
                                        const RowConst& rc) {
  cg::cluster_group cl = cg::this_cluster();
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5, nw = nb >> 5;
  const int P = a.nx >> 5;    // warp separators in the cluster
  const int J = r * nw + wp;  // this warp's separator

  // 1. Poisson law: S_c = sum_{m<=c} (rho_m - rho_bar) dx, E = S - mean(S),
  //    mean(S) = sum_m (nx - m) d_m / nx
  const double d = (w - a.rho_bar) * a.dx;
  double inc = d, t2 = d * rc.wgt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += u;
    t2 += __shfl_xor_sync(kFull, t2, o);
  }
  if (lane == 31) M.wt[wp] = inc;
  if (lane == 0) M.wt[8 + wp] = t2;
  __syncthreads();
  double pw = 0.0;  // the warps before this one
  for (int q = 0; q < wp; ++q) pw += M.wt[q];
  if (tid == 0) {
    double T1 = 0.0, T2 = 0.0;
    for (int q = 0; q < nw; ++q) {
      T1 += M.wt[q];
      T2 += M.wt[8 + q];
    }
    for (int q = 0; q < kCC; ++q) {
      double* e = on_rank(M.ex, q);
      e[2 * r] = T1;
      e[2 * r + 1] = T2;
    }
  }
  cl.sync();
  // every warp combines the CTAs' totals in the same order, so every warp
  // of every CTA holds the same bits: lane q < kCC takes CTA q's totals
  const double x1 = lane < kCC ? M.ex[2 * lane] : 0.0, x2 = lane < kCC ? M.ex[2 * lane + 1] : 0.0;
  double s1 = x1, a1 = x1, a2 = x2;
#pragma unroll
  for (int o = 1; o < kCC; o <<= 1) {
    const double u = __shfl_up_sync(kFull, s1, o);
    if (lane >= o) s1 += u;
    a1 += __shfl_xor_sync(kFull, a1, o);
    a2 += __shfl_xor_sync(kFull, a2, o);
  }
  const double base = __shfl_sync(kFull, s1, (r + kCC - 1) & (kCC - 1));  // CTAs before r (r > 0)
  const double all1 = __shfl_sync(kFull, a1, 0), all2 = __shfl_sync(kFull, a2, 0);
  const double mean = all2 * rc.inv_nx;
  const double E = ((r > 0 ? base : 0.0) + pw + inc) - mean;
  const double E_left = (r > 0 ? base : all1) - mean;  // E at the row before the CTA's first
  M.E[tid] = E;
  __syncthreads();

  // 2. coefficients of row g: lo x_{g-1} + di x_g + up x_{g+1} = rho_g
  const double k = a.m2 * dt * a.inv_dx, idx = a.inv_dx;
  const double El = tid == 0 ? E_left : M.E[tid - 1];
  const double lo = -k * (idx + 0.5 * El);
  const double di = 1.0 - k * (-2.0 * idx - 0.5 * E + 0.5 * El);
  const double up = -k * (idx - 0.5 * E);

  // 3. rows 0..30 of the warp (lane 31, the separator, is an identity row
  //    here): (A, B, C) with right-hand sides D (the data), DL (the
  //    coupling -lo of row 0 to the previous separator) and DR (the
  //    coupling -up of row 30 to this warp's separator).  Parallel cyclic
  //    reduction: at stride o row i takes rows i - o and i + o (identity
  //    rows beyond the warp's ends, where A or C is already zero); after
  //    five strides every row stands alone.
  double A = lane == 0 ? 0.0 : lo, B = di, C = lane == 30 ? 0.0 : up, D = w;
  double DL = lane == 0 ? -lo : 0.0, DR = lane == 30 ? -up : 0.0;
  if (lane == 31) {
    A = 0.0;
    B = 1.0;
    C = 0.0;
    D = 0.0;
    DL = 0.0;
    DR = 0.0;
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double ib = 1.0 / B;
    const double Am = __shfl_up_sync(kFull, A, o), Bm = __shfl_up_sync(kFull, ib, o);
    const double Cm = __shfl_up_sync(kFull, C, o), Dm = __shfl_up_sync(kFull, D, o);
    const double DLm = __shfl_up_sync(kFull, DL, o), DRm = __shfl_up_sync(kFull, DR, o);
    const double Ap = __shfl_down_sync(kFull, A, o), Bp = __shfl_down_sync(kFull, ib, o);
    const double Cp = __shfl_down_sync(kFull, C, o), Dp = __shfl_down_sync(kFull, D, o);
    const double DLp = __shfl_down_sync(kFull, DL, o), DRp = __shfl_down_sync(kFull, DR, o);
    const bool hm = lane >= o, hp = lane + o < 32;
    const double al = hm ? -A * Bm : 0.0, ga = hp ? -C * Bp : 0.0;
    const double nA = hm ? al * Am : 0.0, nC = hp ? ga * Cp : 0.0;
    B = fma(al, hm ? Cm : 0.0, fma(ga, hp ? Ap : 0.0, B));
    D = fma(al, hm ? Dm : 0.0, fma(ga, hp ? Dp : 0.0, D));
    DL = fma(al, hm ? DLm : 0.0, fma(ga, hp ? DLp : 0.0, DL));
    DR = fma(al, hm ? DRm : 0.0, fma(ga, hp ? DRp : 0.0, DR));
    A = nA;
    C = nC;
  }
  const double ib = 1.0 / B;
  // row i = Y + S_{J-1} VL + S_J VR (lanes 0..30)
  const double Y = D * ib, VL = DL * ib, VR = DR * ib;

  // 4. separator J (lane 31, row x31): lo x30 + di x31 + up x32 = rho with
  //    x30 = Y30 + S_{J-1} VL30 + S_J VR30 (this warp) and x32 = Y'0 +
  //    S_J VL'0 + S_{J+1} VR'0 (the next warp's row 0).  Each warp records
  //    its own-side part and its row 0; the system's rows are assembled
  //    from a record and the next one.
  const double Y30 = __shfl_sync(kFull, Y, 30), VL30 = __shfl_sync(kFull, VL, 30);
  const double VR30 = __shfl_sync(kFull, VR, 30);
  double* q = M.rec + 8 * wp;
  if (lane == 31) {
    q[0] = lo * VL30;          // coefficient of S_{J-1}
    q[1] = fma(lo, VR30, di);  // of S_J, this warp's part
    q[2] = fma(-lo, Y30, w);   // right-hand side, this warp's part
    q[3] = up;
  }
  if (lane == 0) {
    q[4] = Y;
    q[5] = VL;
    q[6] = VR;
  }
  cl.sync();
  double sa = 0.0, sb = 1.0, sc = 0.0, sd = 0.0;
  if (lane < P) {  // lane j: separator j
    const int jn = (lane + 1) & (P - 1);
    const double* qj = on_rank(M.rec, lane / nw) + 8 * (lane % nw);
    const double* qn = on_rank(M.rec, jn / nw) + 8 * (jn % nw);
    const double p0 = qj[0], p1 = qj[1], p2 = qj[2], p3 = qj[3];
    const double n4 = qn[4], n5 = qn[5], n6 = qn[6];
    sa = p0;
    sb = fma(p3, n5, p1);
    sc = p3 * n6;
    sd = fma(-p3, n4, p2);
  }
  // cyclic reduction over the P separators (P a power of two): after
  // log2 P strides both couplings of a row point at the row itself
  for (int o = 1; o < P; o <<= 1) {
    const double ib2 = 1.0 / sb;
    const int lm = (lane - o) & (P - 1), lp = (lane + o) & (P - 1);
    const double Am = __shfl_sync(kFull, sa, lm), Bm = __shfl_sync(kFull, ib2, lm);
    const double Cm = __shfl_sync(kFull, sc, lm), Dm = __shfl_sync(kFull, sd, lm);
    const double Ap = __shfl_sync(kFull, sa, lp), Bp = __shfl_sync(kFull, ib2, lp);
    const double Cp = __shfl_sync(kFull, sc, lp), Dp = __shfl_sync(kFull, sd, lp);
    const double al = -sa * Bm, ga = -sc * Bp;
    const double nA = al * Am, nC = ga * Cp;
    sb = fma(al, Cm, fma(ga, Ap, sb));
    sd = fma(al, Dm, fma(ga, Dp, sd));
    sa = nA;
    sc = nC;
  }
  const double S = sd / (sa + sb + sc);

  // 5. the rows from their separators
  const double Sm = __shfl_sync(kFull, S, (J - 1) & (P - 1)), Sj = __shfl_sync(kFull, S, J);
  return lane == 31 ? Sj : fma(Sm, VL, fma(Sj, VR, Y));
}

__device__ double coarse_cluster(const CMap& M, const MacroArgs& a, int nb, int r, double w, const RowConst& rc) {
  const double dt = a.t_span / a.coarse_steps;
  for (int s = 0; s < a.coarse_steps; ++s) w = implicit_step_cluster(M, a, dt, nb, r, w, rc);
  return w;
}

__device__ RowConst row_const(const MacroArgs& a, int g) {
  RowConst rc;
  rc.wgt = (double)(a.nx - g);
  rc.inv_nx = 1.0 / a.nx;
  return rc;
}

// Coarse guess of Algorithm 1 for one solve: rho^{n+1,0} = G(rho^{n,0}).
// blockDim = nb = nx / kCC; thread t of CTA r holds row r nb + t.
__global__ void __launch_bounds__(128) coarse_chain_cluster_kernel(MacroArgs a, int n_slices, double* rho,
                                                                   double* gprev) {
  extern __shared__ __align__(16) double csm[];
  const int nb = a.nx / kCC, r = (int)cg::this_cluster().block_rank(), g = r * nb + threadIdx.x;
  const CMap M = carve_cmap(csm, nb);
  const RowConst rc = row_const(a, g);
  double w = rho[g];
  for (int n = 0; n < n_slices; ++n) {
    w = coarse_cluster(M, a, nb, r, w, rc);
    rho[(size_t)(n + 1) * a.nx + g] = w;
    gprev[(size_t)(n + 1) * a.nx + g] = w;
  }
  cg::this_cluster().sync();  // no CTA leaves while another may read its shared memory
}

// Sequential correction of Algorithm 1 for one solve, n = k..N-1:
// Gn = G(rho^{n,k+1}); rho^{n+1,k+1} = F + (Gn - Gprev); Gprev = Gn; and the
// successive error max |rho^{n+1,k+1} - rho^{n+1,k}|.
__global__ void __launch_bounds__(128) correct_cluster_kernel(CorrectArgs c) {
  extern __shared__ __align__(16) double csm[];
  const MacroArgs& a = c.m;
  const int nx = a.nx, nb = nx / kCC, r = (int)cg::this_cluster().block_rank(), g = r * nb + threadIdx.x;
  const CMap M = carve_cmap(csm, nb);
  const RowConst rc = row_const(a, g);
  double w = c.rho[(size_t)c.k * nx + g];
  double emax = 0.0;
  for (int n = c.k; n < c.n_slices; ++n) {
    const double gn = coarse_cluster(M, a, nb, r, w, rc);
    const size_t at = (size_t)(n + 1) * nx + g;
    const double v = c.frho[at] + (gn - c.gprev[at]);
    emax = fmax(emax, fabs(v - c.rho[at]));
    c.rho[at] = v;
    c.gprev[at] = gn;
    w = v;
  }
  for (int m = 16; m > 0; m >>= 1) emax = fmax(emax, __shfl_xor_sync(kFull, emax, m));
  if ((threadIdx.x & 31) == 0) M.wt[threadIdx.x >> 5] = emax;  // the totals are dead after the last step
  __syncthreads();
  if (threadIdx.x == 0) {
    double e = 0.0;
    for (int q = 0; q < nb / 32; ++q) e = fmax(e, M.wt[q]);
    on_rank(M.em, 0)[r] = e;  // rank 0 gathers the CTAs' maxima
  }
  cg::this_cluster().sync();
  if (r == 0 && threadIdx.x == 0) {
    double e = 0.0;
    for (int q = 0; q < kCC; ++q) e = fmax(e, M.em[q]);
    *c.err = e;
  }
}

template <class K, class... Args>
cudaError_t launch_cluster(K kernel, int nb, cudaStream_t s, Args... args) {
  const size_t smem = cmap_doubles(nb) * sizeof(double);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCC);
  cfg.blockDim = dim3(nb);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kCC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

bool coarse_cluster_ok(const MacroArgs& a) {
  // one row per thread and a whole number of warps per CTA (nx >= 256);
  // the warp separators (nx / 32) in one warp's lanes (nx <= 1024); nx a
  // power of two for the cyclic reduction over them
  const int nx = a.nx;
  return a.coarse_kind == 0 && nx >= 32 * kCC && nx <= 32 * 32 && (nx & (nx - 1)) == 0;
}

cudaError_t launch_coarse_chain_cluster(const MacroArgs& a, int n_slices, double* rho, double* gprev,
                                        cudaStream_t s) {
  return launch_cluster(coarse_chain_cluster_kernel, a.nx / kCC, s, a, n_slices, rho, gprev);
}

cudaError_t launch_correct_cluster(const CorrectArgs& c, cudaStream_t s) {
  return launch_cluster(correct_cluster_kernel, c.m.nx / kCC, s, c);
}

}  // namespace mmk
