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
//   - T = min(nx / kCC, 128) threads per CTA (one warp per sub-partition),
//     thread t of CTA r owning the m = nx / (kCC T) consecutive rows
//     [r nb + t m, r nb + t m + m), nb = m T, the last of them the
//     thread's separator;
//   - with m > 1 each thread eliminates its m - 1 interior rows by a Thomas
//     sweep with three right-hand sides (the data and the couplings to the
//     previous thread's separator and its own), which leaves one reduced
//     row per thread between neighbouring separators;
//   - each warp eliminates its 31 interior separators by parallel cyclic
//     reduction in registers (shuffles, no barrier), again with the data
//     and the couplings to its two bounding warp separators (the previous
//     warp's last separator and its own);
//   - the kCC T / 32 warp separators form a cyclic tridiagonal system that
//     every warp assembles from the records of all warps (one exchange
//     through distributed shared memory) and solves redundantly by
//     parallel cyclic reduction in registers;
//   - every separator, then every interior row, is rebuilt from the two
//     separators that bound it.
// Two cluster barriers per step, against one per reduction level when the
// reduction itself is distributed over the cluster: about 11 us per step at
// Nx = 1024 against 16 us for that layout.
//
// Per step:
//   1. the Poisson law of S^MM for the frozen field: per-thread sums of the
//      density deviations, a warp scan, the warps' totals through shared
//      memory, the CTAs' totals through distributed shared memory;
//   2. the coefficients of (I - m2 dt L_E) x = rho, and with m > 1 the
//      interior rows' elimination;
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

// Shared memory of one CTA (doubles).  The per-row arrays of the chunked
// layout (m > 1) are interleaved, row j of thread t at j T + t, so that a
// warp's 32 threads touch 32 consecutive words.
struct CMap {
  double* E;    // [T] field at each thread's last row
  double* rec;  // [T / 32][8] separator record of each warp
  double* ex;   // [kCC][2] the CTAs' Poisson totals (pushed by every CTA)
  double* wt;   // [2][8] the warps' Poisson totals
  double* em;   // [kCC] the CTAs' maximum corrections (rank 0's copy)
  double *W, *CW, *Y, *VL, *VR;  // [m][T] (m > 1): density, and the
                                 // interior rows' elimination
};

__host__ __device__ inline size_t cmap_doubles(int T, int m) {
  return (size_t)T + 8 * (T / 32) + 2 * kCC + 16 + kCC + (m > 1 ? (size_t)5 * m * T : 0);
}

__device__ CMap carve_cmap(double* base, int T, int m) {
  CMap c;
  c.E = base;
  c.rec = c.E + T;
  c.ex = c.rec + 8 * (T / 32);
  c.wt = c.ex + 2 * kCC;
  c.em = c.wt + 16;
  double* q = c.em + kCC;
  const size_t n = m > 1 ? (size_t)m * T : 0;
  c.W = q;
  c.CW = q + n;
  c.Y = q + 2 * n;
  c.VL = q + 3 * n;
  c.VR = q + 4 * n;
  return c;
}

// Launch shape of one solve: threads per CTA and rows per thread.
__host__ __device__ inline int cluster_threads(int nx) { return nx / kCC < 128 ? nx / kCC : 128; }
__host__ __device__ inline int cluster_rows(int nx) { return nx / (kCC * cluster_threads(nx)); }

// Per-thread constants of a chain: the weight nx - g of the thread's first
// row in the mean of the Poisson prefix sums, and 1 / nx.
struct RowConst {
  double wgt, inv_nx;
};

// Coefficients of row i: lo x_{i-1} + di x_i + up x_{i+1} = rho_i with the
// field El at interface i - 1/2 and Er at i + 1/2.
__device__ __forceinline__ void coef(const MacroArgs& a, double k, double El, double Er, double& lo, double& di,
                                     double& up) {
  const double idx = a.inv_dx;
  lo = -k * (idx + 0.5 * El);
  di = 1.0 - k * (-2.0 * idx - 0.5 * Er + 0.5 * El);
  up = -k * (idx - 0.5 * Er);
}

// One linearly implicit S^0 step of the cluster's density, (I - m2 dt
// L_E) x = rho with E frozen from rho.  CHUNK = false: one row per thread,
// held in w (returned updated); CHUNK = true: m rows per thread in M.W
// (updated in place; w unused).
template <bool CHUNK>
__device__ double implicit_step_cluster(const CMap& M, const MacroArgs& a, double dt, int m, int r, double w,
                                        const RowConst& rc) {
  cg::cluster_group cl = cg::this_cluster();
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wp = tid >> 5, nw = T >> 5;
  const int P = kCC * nw;     // warp separators in the cluster
  const int J = r * nw + wp;  // this warp's separator

  // 1. Poisson law: S_c = sum_{m<=c} (rho_m - rho_bar) dx, E = S - mean(S),
  //    mean(S) = sum_m (nx - m) d_m / nx
  double tsum, t2;
  if constexpr (!CHUNK) {
    tsum = (w - a.rho_bar) * a.dx;
    t2 = tsum * rc.wgt;
  } else {
    tsum = 0.0;
    t2 = 0.0;
    double wg = rc.wgt;
    for (int j = 0; j < m; ++j) {
      const double d = (M.W[j * T + tid] - a.rho_bar) * a.dx;
      tsum += d;
      t2 += d * wg;
      wg -= 1.0;
    }
  }
  double inc = tsum;
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
  const double E_left = (r > 0 ? base : all1) - mean;  // E at the row before the CTA's first
  const double k = a.m2 * dt * a.inv_dx;

  // 2. this thread's separator row in terms of its neighbours, a s_{t-1} +
  //    b s_t + c s_{t+1} = d; with m > 1 after the Thomas sweep of the
  //    interior rows, x_j = y_j + s_{t-1} vl_j + s_t vr_j.  b_own, d_own:
  //    the parts that do not involve the next thread (the record of a
  //    warp's last thread carries them).
  double a_, b_own, d_own, b_, c_, d_, up_s;
  double yF = 0.0, vlF = 0.0, vrF = 0.0;  // first interior row (m > 1)
  if constexpr (!CHUNK) {
    const double E = ((r > 0 ? base : 0.0) + pw + inc) - mean;
    M.E[tid] = E;
    __syncthreads();
    const double El = tid == 0 ? E_left : M.E[tid - 1];
    double lo, di, up;
    coef(a, k, El, E, lo, di, up);
    a_ = lo;
    b_own = b_ = di;
    c_ = up_s = up;
    d_own = d_ = w;
  } else {
    const double excl0 = __shfl_up_sync(kFull, inc, 1);
    const double excl = lane > 0 ? excl0 : 0.0;
    const double Sb = ((r > 0 ? base : 0.0) + pw) + excl;  // S at the row before the chunk
    M.E[tid] = (Sb + tsum) - mean;
    __syncthreads();
    double Eprev = tid == 0 ? E_left : M.E[tid - 1];
    double run = 0.0, cprev = 0.0, yp = 0.0, lp = 0.0, rp = 0.0;
    for (int j = 0; j < m - 1; ++j) {  // forward sweep over the interior rows
      const int at = j * T + tid;
      const double wj = M.W[at];
      run += (wj - a.rho_bar) * a.dx;
      const double Ej = (Sb + run) - mean;
      double lo, di, up;
      coef(a, k, Eprev, Ej, lo, di, up);
      const double l = j == 0 ? 0.0 : lo;
      const double inv = 1.0 / (di - l * cprev);
      cprev = j == m - 2 ? 0.0 : up * inv;
      yp = (wj - l * yp) * inv;
      lp = ((j == 0 ? -lo : 0.0) - l * lp) * inv;
      rp = j == m - 2 ? -up * inv : 0.0;
      M.CW[at] = cprev;
      M.Y[at] = yp;
      M.VL[at] = lp;
      M.VR[at] = rp;
      Eprev = Ej;
    }
    const double yL = yp, vlL = lp, vrL = rp;  // the last interior row, final
    for (int j = m - 3; j >= 0; --j) {  // back substitution
      const int at = j * T + tid;
      const double cw = M.CW[at];
      yp = M.Y[at] - cw * yp;
      lp = M.VL[at] - cw * lp;
      rp = M.VR[at] - cw * rp;
      M.Y[at] = yp;
      M.VL[at] = lp;
      M.VR[at] = rp;
    }
    yF = yp;
    vlF = lp;
    vrF = rp;
    // the separator row (j = m - 1)
    const double ws = M.W[(m - 1) * T + tid];
    run += (ws - a.rho_bar) * a.dx;
    const double Es = (Sb + run) - mean;
    double lo, di;
    coef(a, k, Eprev, Es, lo, di, up_s);
    a_ = lo * vlL;
    b_own = fma(lo, vrL, di);
    d_own = fma(-lo, yL, ws);
    // the next thread's first interior row (its couplings: s_t and s_{t+1})
    const double yFn = __shfl_down_sync(kFull, yF, 1), vlFn = __shfl_down_sync(kFull, vlF, 1);
    const double vrFn = __shfl_down_sync(kFull, vrF, 1);
    b_ = fma(up_s, vlFn, b_own);
    c_ = up_s * vrFn;
    d_ = fma(-up_s, yFn, d_own);
  }

  // 3. separators 0..30 of the warp (lane 31, the warp's separator, is an
  //    identity row here): (A, B, C) with right-hand sides D (the data), DL
  //    (the coupling -a of separator 0 to the previous warp's separator)
  //    and DR (the coupling -c of separator 30 to this warp's).  Parallel
  //    cyclic reduction: at stride o row i takes rows i - o and i + o
  //    (identity rows beyond the warp's ends, where A or C is already
  //    zero); after five strides every row stands alone.
  double A = lane == 0 ? 0.0 : a_, B = b_, C = lane == 30 ? 0.0 : c_, D = d_;
  double DL = lane == 0 ? -a_ : 0.0, DR = lane == 30 ? -c_ : 0.0;
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
  // separator t = Y + S_{J-1} VL + S_J VR (lanes 0..30)
  const double Y = D * ib, VL = DL * ib, VR = DR * ib;

  // 4. warp separator J (lane 31): a s30 + b_own S_J + up x' = d_own, with
  //    s30 = Y30 + S_{J-1} VL30 + S_J VR30 from this warp and x' the next
  //    warp's first row (m = 1: its separator 0; m > 1: its thread 0's first
  //    interior row), x' = e0 + S_J e1 + S_{J+1} e2.  Each warp records its
  //    own-side part and its e; the system's rows are assembled from a
  //    record and the next one.
  const double Y30 = __shfl_sync(kFull, Y, 30), VL30 = __shfl_sync(kFull, VL, 30);
  const double VR30 = __shfl_sync(kFull, VR, 30);
  double* q = M.rec + 8 * wp;
  if (lane == 31) {
    q[0] = a_ * VL30;             // coefficient of S_{J-1}
    q[1] = fma(a_, VR30, b_own);  // of S_J, this warp's part
    q[2] = fma(-a_, Y30, d_own);  // right-hand side, this warp's part
    q[3] = up_s;
  }
  if (lane == 0) {
    if constexpr (!CHUNK) {
      q[4] = Y;
      q[5] = VL;
      q[6] = VR;
    } else {
      q[4] = fma(vrF, Y, yF);
      q[5] = fma(vrF, VL, vlF);
      q[6] = vrF * VR;
    }
  }
  cl.sync();
  double sa = 0.0, sb = 1.0, sc = 0.0, sd = 0.0;
  if (lane < P) {  // lane j: warp separator j
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
  // cyclic reduction over the P warp separators (P a power of two): after
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

  // 5. the separators, then the interior rows, from the separators that
  //    bound them
  const double Sm = __shfl_sync(kFull, S, (J - 1) & (P - 1)), Sj = __shfl_sync(kFull, S, J);
  const double st = lane == 31 ? Sj : fma(Sm, VL, fma(Sj, VR, Y));
  if constexpr (!CHUNK) {
    return st;
  } else {
    const double sp0 = __shfl_up_sync(kFull, st, 1);
    const double sprev = lane == 0 ? Sm : sp0;
    for (int j = 0; j < m - 1; ++j) {
      const int at = j * T + tid;
      M.W[at] = fma(sprev, M.VL[at], fma(st, M.VR[at], M.Y[at]));
    }
    M.W[(m - 1) * T + tid] = st;
    return 0.0;
  }
}

template <bool CHUNK>
__device__ double coarse_cluster(const CMap& M, const MacroArgs& a, int m, int r, double w, const RowConst& rc) {
  const double dt = a.t_span / a.coarse_steps;
  for (int s = 0; s < a.coarse_steps; ++s) w = implicit_step_cluster<CHUNK>(M, a, dt, m, r, w, rc);
  return w;
}

// One solve's rows of this thread: m, the first row g0 and its constants.
struct Rows {
  int m, T, r, g0;
  RowConst rc;
};

template <bool CHUNK>
__device__ Rows rows_of(const MacroArgs& a) {
  Rows q;
  q.T = blockDim.x;
  q.m = CHUNK ? cluster_rows(a.nx) : 1;
  q.r = (int)cg::this_cluster().block_rank();
  q.g0 = q.r * q.m * q.T + (int)threadIdx.x * q.m;
  q.rc.wgt = (double)(a.nx - q.g0);
  q.rc.inv_nx = 1.0 / a.nx;
  return q;
}

// Coarse guess of Algorithm 1 for one solve: rho^{n+1,0} = G(rho^{n,0}),
// Gprev = rho^{n+1,0}.
template <bool CHUNK>
__device__ void chain_body(const MacroArgs& a, int n_slices, double* rho, double* gprev, double* csm) {
  const Rows q = rows_of<CHUNK>(a);
  const CMap M = carve_cmap(csm, q.T, q.m);
  double w = 0.0;
  if constexpr (!CHUNK) w = rho[q.g0];
  else
    for (int j = 0; j < q.m; ++j) M.W[j * q.T + threadIdx.x] = rho[q.g0 + j];
  for (int n = 0; n < n_slices; ++n) {
    w = coarse_cluster<CHUNK>(M, a, q.m, q.r, w, q.rc);
    const size_t at = (size_t)(n + 1) * a.nx + q.g0;
    if constexpr (!CHUNK) {
      rho[at] = w;
      gprev[at] = w;
    } else {
      for (int j = 0; j < q.m; ++j) {
        const double v = M.W[j * q.T + threadIdx.x];
        rho[at + j] = v;
        gprev[at + j] = v;
      }
    }
  }
  cg::this_cluster().sync();  // no CTA leaves while another may read its shared memory
}

// Sequential correction of Algorithm 1 for one solve, n = k..N-1:
// Gn = G(rho^{n,k+1}); rho^{n+1,k+1} = F + (Gn - Gprev); Gprev = Gn; and the
// successive error max |rho^{n+1,k+1} - rho^{n+1,k}|.
template <bool CHUNK>
__device__ void correct_body(const CorrectArgs& c, double* csm) {
  const MacroArgs& a = c.m;
  const int nx = a.nx;
  const Rows q = rows_of<CHUNK>(a);
  const CMap M = carve_cmap(csm, q.T, q.m);
  double w = 0.0;
  const size_t k0 = (size_t)c.k * nx + q.g0;
  if constexpr (!CHUNK) w = c.rho[k0];
  else
    for (int j = 0; j < q.m; ++j) M.W[j * q.T + threadIdx.x] = c.rho[k0 + j];
  double emax = 0.0;
  for (int n = c.k; n < c.n_slices; ++n) {
    const double gw = coarse_cluster<CHUNK>(M, a, q.m, q.r, w, q.rc);
    const size_t at = (size_t)(n + 1) * nx + q.g0;
    for (int j = 0; j < q.m; ++j) {
      const int sj = j * q.T + (int)threadIdx.x;
      const double gn = CHUNK ? M.W[sj] : gw;
      const double v = c.frho[at + j] + (gn - c.gprev[at + j]);
      emax = fmax(emax, fabs(v - c.rho[at + j]));
      c.rho[at + j] = v;
      c.gprev[at + j] = gn;
      if constexpr (CHUNK) M.W[sj] = v;
      else w = v;
    }
  }
  for (int s = 16; s > 0; s >>= 1) emax = fmax(emax, __shfl_xor_sync(kFull, emax, s));
  if ((threadIdx.x & 31) == 0) M.wt[threadIdx.x >> 5] = emax;  // the totals are dead after the last step
  __syncthreads();
  if (threadIdx.x == 0) {
    double e = 0.0;
    for (int w8 = 0; w8 < q.T / 32; ++w8) e = fmax(e, M.wt[w8]);
    on_rank(M.em, 0)[q.r] = e;  // rank 0 gathers the CTAs' maxima
  }
  cg::this_cluster().sync();
  if (q.r == 0 && threadIdx.x == 0) {
    double e = 0.0;
    for (int r = 0; r < kCC; ++r) e = fmax(e, M.em[r]);
    *c.err = e;
  }
}

template <bool CHUNK>
__global__ void __launch_bounds__(128) coarse_chain_cluster_kernel(MacroArgs a, int n_slices, double* rho,
                                                                   double* gprev) {
  extern __shared__ __align__(16) double csm[];
  chain_body<CHUNK>(a, n_slices, rho, gprev, csm);
}

template <bool CHUNK>
__global__ void __launch_bounds__(128) correct_cluster_kernel(CorrectArgs c) {
  extern __shared__ __align__(16) double csm[];
  correct_body<CHUNK>(c, csm);
}

// The same for many solves of one grid size, one cluster each.
template <bool CHUNK>
__global__ void __launch_bounds__(128) coarse_chain_cluster_list_kernel(const CorrectArgs* list) {
  extern __shared__ __align__(16) double csm[];
  const CorrectArgs& c = list[blockIdx.x / kCC];
  chain_body<CHUNK>(c.m, c.n_slices, c.rho, c.gprev, csm);
}

template <bool CHUNK>
__global__ void __launch_bounds__(128) correct_cluster_list_kernel(const CorrectArgs* list) {
  extern __shared__ __align__(16) double csm[];
  correct_body<CHUNK>(list[blockIdx.x / kCC], csm);
}

template <class K, class... Args>
cudaError_t launch_cluster(K kernel, int nx, int n_clusters, cudaStream_t s, Args... args) {
  const int T = cluster_threads(nx);
  const size_t smem = cmap_doubles(T, cluster_rows(nx)) * sizeof(double);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCC * n_clusters);
  cfg.blockDim = dim3(T);
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
  // a whole number of warps per CTA (nx >= 256), at most 32 warp
  // separators (kCC x 4 warps), nx a power of two for the cyclic reduction
  // over them, and at most 32 rows per thread (the chunked layout's
  // 5 m T doubles of shared memory: 160 KB at nx = 32768)
  const int nx = a.nx;
  return a.coarse_kind == 0 && nx >= 32 * kCC && nx <= 32768 && (nx & (nx - 1)) == 0;
}

cudaError_t launch_coarse_chain_cluster(const MacroArgs& a, int n_slices, double* rho, double* gprev,
                                        cudaStream_t s) {
  if (cluster_rows(a.nx) > 1)
    return launch_cluster(coarse_chain_cluster_kernel<true>, a.nx, 1, s, a, n_slices, rho, gprev);
  return launch_cluster(coarse_chain_cluster_kernel<false>, a.nx, 1, s, a, n_slices, rho, gprev);
}

cudaError_t launch_correct_cluster(const CorrectArgs& c, cudaStream_t s) {
  if (cluster_rows(c.m.nx) > 1) return launch_cluster(correct_cluster_kernel<true>, c.m.nx, 1, s, c);
  return launch_cluster(correct_cluster_kernel<false>, c.m.nx, 1, s, c);
}

cudaError_t launch_coarse_chain_cluster_list(const CorrectArgs* list, int n, int nx, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (cluster_rows(nx) > 1) return launch_cluster(coarse_chain_cluster_list_kernel<true>, nx, n, s, list);
  return launch_cluster(coarse_chain_cluster_list_kernel<false>, nx, n, s, list);
}

cudaError_t launch_correct_cluster_list(const CorrectArgs* list, int n, int nx, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (cluster_rows(nx) > 1) return launch_cluster(correct_cluster_list_kernel<true>, nx, n, s, list);
  return launch_cluster(correct_cluster_list_kernel<false>, nx, n, s, list);
}

}  // namespace mmk
