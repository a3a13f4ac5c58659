// Coarse propagator G = S^0 (Sec. 2.3), lifting of order one (Def. 1,
// Sec. 3.2-3.3) and the device side of Algorithm 1: the coarse guess, the
// sequential correction sweep and the successive error.  All in double
// (the correction and the convergence test of the parareal loop stay in
// double precision in both precisions of the fine propagator).
//
// One CTA of 256 threads owns one density; the linearly implicit step
// solves the cyclic tridiagonal system (I - m2 dt L_E) rho^{m+1} = rho^m
// with E frozen from rho^m by a partitioned solve: Thomas sweeps over
// chunks of about 8 rows in parallel, parallel cyclic reduction on the
// chunk separators (the system is strictly diagonally dominant for the
// slice lengths used, so no pivoting is needed).  FP64 latency on GB300
// (~70 cycles per dependent add or FMA, ~600 per division) makes the length
// of the serial chains, not the operation count, the cost.
#include <math.h>

#include "lift.cuh"
#include "mm_internal.h"

namespace mmk {

constexpr int kMacroThreads = 256;

// Block-wide Poisson law of S^MM: E_{i+1/2} = S_i - mean(S),
// S_i = sum_{m<=i} (rho_m - rho_bar) dx.  red: >= 64 doubles of smem.
__device__ void poisson_block(const double* rho, double* E, int nx, double rho_bar, double dx,
                              double* red) {
  const int T = blockDim.x, tid = threadIdx.x;
  const int cpt = (nx + T - 1) / T;
  const int c0 = min(tid * cpt, nx), c1 = min(c0 + cpt, nx);
  double t1 = 0.0, t2 = 0.0;
  for (int c = c0; c < c1; ++c) {
    const double d = (rho[c] - rho_bar) * dx;
    t1 += d;
    E[c] = t1;
    t2 += d * (double)(nx - c);
  }
  const int w = tid >> 5, l = tid & 31;
  double inc = t1;
  for (int d = 1; d < 32; d <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, inc, d);
    if (l >= d) inc += t;
  }
  double excl_w = __shfl_up_sync(0xffffffffu, inc, 1);
  if (l == 0) excl_w = 0.0;
  double ws = t2;
  for (int m = 16; m > 0; m >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, m);
  __syncthreads();
  if (l == 31) red[w] = inc;
  if (l == 0) red[32 + w] = ws;
  __syncthreads();
  double off = 0.0, tw = 0.0;
  for (int q = 0; q < (T >> 5); ++q) {
    if (q < w) off += red[q];
    tw += red[32 + q];
  }
  const double mean = tw * (1.0 / nx);
  const double base = off + excl_w;
  for (int c = c0; c < c1; ++c) E[c] = base + E[c] - mean;
  __syncthreads();
}

// One explicit S^0 step, in place.
__device__ void limit_step_block(double* rho, double* E, double* J, const MacroArgs& a, double dt,
                                 double* red) {
  const int nx = a.nx, T = blockDim.x;
  poisson_block(rho, E, nx, a.rho_bar, a.dx, red);
  for (int i = threadIdx.x; i < nx; i += T) {
    const double r0 = rho[i], r1 = rho[i + 1 == nx ? 0 : i + 1];
    J[i] = (r1 - r0) * a.inv_dx - E[i] * 0.5 * (r0 + r1);
  }
  __syncthreads();
  const double k = a.m2 * dt * a.inv_dx;
  for (int i = threadIdx.x; i < nx; i += T) rho[i] += k * (J[i] - J[i == 0 ? nx - 1 : i - 1]);
  __syncthreads();
}

// Cyclic tridiagonal system of P rows (P a power of two, <= blockDim.x),
// row i: A_i x_{i-1} + B_i x_i + C_i x_{i+1} = D_i (indices mod P), by
// parallel cyclic reduction: at stride s every row eliminates its
// neighbours at distance s, so after log2(P) levels row i couples x_i only
// with x_{i +- P} = x_i itself.  One reciprocal per row and level (FP64
// divisions are ~600 cycles on this GPU; the chain is log2(P) levels deep
// instead of P rows).  A, B, C, D are overwritten; x receives the solution.
__device__ void pcr_cyclic(int P, double* A, double* B, double* C, double* D, double* x) {
  const int i = threadIdx.x;
  double a = 0, b = 1, c = 0, d = 0;
  if (i < P) {
    a = A[i];
    b = B[i];
    c = C[i];
    d = D[i];
  }
  for (int st = 1; st < P; st <<= 1) {
    __syncthreads();
    if (i < P) {  // publish this level: B holds 1/b
      A[i] = a;
      B[i] = 1.0 / b;
      C[i] = c;
      D[i] = d;
    }
    __syncthreads();
    if (i < P) {
      const int im = (i - st) & (P - 1), ip = (i + st) & (P - 1);
      const double al = -a * B[im], ga = -c * B[ip];
      const double na = al * A[im], nc = ga * C[ip];
      b = fma(al, C[im], fma(ga, A[ip], b));
      d = fma(al, D[im], fma(ga, D[ip], d));
      a = na;
      c = nc;
    }
  }
  if (i < P) x[i] = d / (a + b + c);
  __syncthreads();
}

// One linearly implicit S^0 step, in place: (I - m2 dt L_E) x = rho with E
// frozen from rho.  Partitioned solve: the rows are cut into P chunks whose
// last row is a separator; thread p eliminates the interior of chunk p
// (Thomas, three right-hand sides: the data and the couplings to the two
// neighbouring separators), the separators satisfy a cyclic P x P
// tridiagonal system (parallel cyclic reduction), then every chunk is
// rebuilt.  Scratch: E, cw, y, vl, vr (nx each) and rs (>= 7 * 256 doubles).
__device__ void limit_step_implicit_block(double* rho, double* E, double* cw, double* y, double* vl,
                                          double* vr, double* rs, const MacroArgs& a, double dt,
                                          double* red) {
  const int n = a.nx, P = a.parts, tid = threadIdx.x;
  poisson_block(rho, E, n, a.rho_bar, a.dx, red);
  const double k = a.m2 * dt * a.inv_dx, idx = a.inv_dx;
  auto coef = [&](int i, double& lo, double& di, double& up) {
    const double Er = E[i], El = E[i == 0 ? n - 1 : i - 1];
    lo = -k * (idx + 0.5 * El);
    di = 1.0 - k * (-2.0 * idx - 0.5 * Er + 0.5 * El);
    up = -k * (idx - 0.5 * Er);
  };
  if (tid < P) {  // interior rows [a0, b0) of chunk tid; separator b0
    const int a0 = (int)(((long long)tid * n) / P), b0 = (int)(((long long)(tid + 1) * n) / P) - 1;
    double lo, di, up, cprev = 0.0, yp = 0.0, lp = 0.0, rp = 0.0;
    for (int i = a0; i < b0; ++i) {
      coef(i, lo, di, up);
      const double l = (i == a0) ? 0.0 : lo;
      const double inv = 1.0 / (di - l * cprev);
      cprev = (i == b0 - 1) ? 0.0 : up * inv;
      cw[i] = cprev;
      yp = (rho[i] - l * yp) * inv;
      lp = ((i == a0 ? -lo : 0.0) - l * lp) * inv;
      // the right coupling enters at the chunk's last interior row only;
      // before it the forward sweep of that column is zero
      rp = (i == b0 - 1) ? -up * inv : 0.0;
      y[i] = yp;
      vl[i] = lp;
      vr[i] = rp;
    }
    for (int i = b0 - 2; i >= a0; --i) {
      y[i] -= cw[i] * y[i + 1];
      vl[i] -= cw[i] * vl[i + 1];
      vr[i] -= cw[i] * vr[i + 1];
    }
  }
  __syncthreads();
  double* rA = rs;          // reduced system on the separators
  double* rB = rs + 256;
  double* rC = rs + 512;
  double* rD = rs + 768;
  double* rL = rs + 1024;
  if (tid < P) {
    const int b0 = (int)(((long long)(tid + 1) * n) / P) - 1;
    const int il = b0 - 1, ir = (b0 + 1 == n) ? 0 : b0 + 1;
    double lo, di, up;
    coef(b0, lo, di, up);
    rA[tid] = lo * vl[il];
    rB[tid] = lo * vr[il] + di + up * vl[ir];
    rC[tid] = up * vr[ir];
    rD[tid] = rho[b0] - lo * y[il] - up * y[ir];
  }
  __syncthreads();
  pcr_cyclic(P, rA, rB, rC, rD, rL);
  if (tid < P) {
    const int a0 = (int)(((long long)tid * n) / P), b0 = (int)(((long long)(tid + 1) * n) / P) - 1;
    const double Lm = rL[tid == 0 ? P - 1 : tid - 1], Lp = rL[tid];
    for (int i = a0; i < b0; ++i) rho[i] = y[i] + Lm * vl[i] + Lp * vr[i];
    rho[b0] = Lp;
  }
  __syncthreads();
}

// Per-CTA scratch: the density working copy, five arrays of nx doubles and
// the reduced system, in dynamic shared memory when they fit, else in a
// global workspace.
constexpr int kScratchArrays = 6;
constexpr int kReducedDoubles = 7 * 256;

struct Scratch {
  double *w, *s0, *s1, *s2, *s3, *s4, *rs;
};

__device__ Scratch scratch_of(unsigned char* smem, double* gws, int nx, int in_smem, size_t per = 0) {
  if (per == 0) per = (size_t)kScratchArrays * nx + kReducedDoubles;
  double* base = in_smem ? reinterpret_cast<double*>(smem + 1024) : gws + (size_t)blockIdx.x * per;
  return {base, base + nx, base + 2 * nx, base + 3 * nx, base + 4 * nx, base + 5 * nx, base + 6 * nx};
}

// G over a span, in place (kind 0: implicit, 1: explicit).
__device__ void coarse_block(const Scratch& S, const MacroArgs& a, double* red) {
  const double dt = a.t_span / a.coarse_steps;
  for (int s = 0; s < a.coarse_steps; ++s) {
    if (a.coarse_kind == 0) limit_step_implicit_block(S.w, S.s0, S.s1, S.s2, S.s3, S.s4, S.rs, a, dt, red);
    else limit_step_block(S.w, S.s0, S.s1, a, dt, red);
  }
}

__global__ void coarse_kernel(MacroArgs a, const double* rho_in, double* rho_out, double* gws,
                              int in_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = reinterpret_cast<double*>(smem);
  const int nx = a.nx;
  Scratch S = scratch_of(smem, gws, nx, in_smem);
  const double* ri = rho_in + (size_t)blockIdx.x * nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) S.w[i] = ri[i];
  __syncthreads();
  coarse_block(S, a, red);
  double* ro = rho_out + (size_t)blockIdx.x * nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) ro[i] = S.w[i];
}

template <class G>
__global__ void lift_kernel(MacroArgs a, const double* rho, G* g, double* gws, int in_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = reinterpret_cast<double*>(smem);
  const int nx = a.nx, nv = a.nv;
  Scratch S = scratch_of(smem, gws, nx, in_smem);
  const double* ri = rho + (size_t)blockIdx.x * nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) S.w[i] = ri[i];
  __syncthreads();
  poisson_block(S.w, S.s0, nx, a.rho_bar, a.dx, red);
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double r0 = S.w[i], r1 = S.w[i + 1 == nx ? 0 : i + 1];
    S.s1[i] = (r1 - r0) * a.inv_dx - S.s0[i] * 0.5 * (r0 + r1);
  }
  __syncthreads();
  const double* vM = a.vtab + 2 * nv;  // v_j M_j
  const double* Mj = a.vtab + 1 * nv;
  const double* vj = a.vtab + 5 * nv;
  G* gb = g + (size_t)blockIdx.x * nx * nv;
  const size_t n = (size_t)nx * nv;
  if (a.lift_order <= 1) {  // g = -eps (xi_j M_j - <xi M> M_j) J_i
    for (size_t q = threadIdx.x; q < n; q += blockDim.x) {
      const int i = (int)(q / nv), j = (int)(q % nv);
      const double J = S.s1[i];
      gb[q] = (G)(-a.eps * (vM[j] * J - a.xiM * J * Mj[j]));
    }
    return;
  }
  // orders two and three: K -> s4, dK -> s2, dtJ -> s3
  lift_fields(S.w, S.s0, S.s1, S.s4, S.s2, S.s3, nx, a.inv_dx, red);
  const LiftConsts lc{a.lift_order, a.eps, a.xiM, a.m2, a.mu3};
  for (size_t q = threadIdx.x; q < n; q += blockDim.x) {
    const int i = (int)(q / nv), j = (int)(q % nv);
    gb[q] = (G)lift_value(lc, vj[j], Mj[j], S.s0[i], S.s1[i], S.s4[i], S.s2[i], S.s3[i]);
  }
}

// Lifted difference of the full-state correction, one CTA per slice:
// g[b] += L rho_new[b] - L rho_old[b] (lifting of order a.lift_order).  Both
// liftings are formed in double and subtracted before the addition, so a
// slice whose coarse value did not change keeps its fine g bitwise.  ws: 12
// arrays of nx doubles per CTA in global memory.
template <class G>
__global__ void lift_diff_kernel(MacroArgs a, const double* rho_new, const double* rho_old, G* g, double* ws) {
  __shared__ double red[64];
  const int nx = a.nx, nv = a.nv, T = blockDim.x;
  double* base = ws + (size_t)blockIdx.x * 12 * nx;
  double* R[2] = {base, base + 6 * nx};  // rho, E, J, K, dK, dtJ per density
  const double* src[2] = {rho_new + (size_t)blockIdx.x * nx, rho_old + (size_t)blockIdx.x * nx};
  for (int d = 0; d < 2; ++d) {
    double* rho = R[d];
    double* E = rho + nx;
    double* J = rho + 2 * nx;
    for (int i = threadIdx.x; i < nx; i += T) rho[i] = src[d][i];
    __syncthreads();
    poisson_block(rho, E, nx, a.rho_bar, a.dx, red);
    for (int i = threadIdx.x; i < nx; i += T) {
      const double r0 = rho[i], r1 = rho[i + 1 == nx ? 0 : i + 1];
      J[i] = (r1 - r0) * a.inv_dx - E[i] * 0.5 * (r0 + r1);
    }
    __syncthreads();
    if (a.lift_order >= 2) lift_fields(rho, E, J, rho + 3 * nx, rho + 4 * nx, rho + 5 * nx, nx, a.inv_dx, red);
  }
  const double* vM = a.vtab + 2 * nv;
  const double* Mj = a.vtab + 1 * nv;
  const double* vj = a.vtab + 5 * nv;
  const LiftConsts lc{a.lift_order, a.eps, a.xiM, a.m2, a.mu3};
  G* gb = g + (size_t)blockIdx.x * nx * nv;
  const size_t n = (size_t)nx * nv;
  for (size_t q = threadIdx.x; q < n; q += T) {
    const int i = (int)(q / nv), j = (int)(q % nv);
    double l[2];
    for (int d = 0; d < 2; ++d) {
      const double* rho = R[d];
      if (a.lift_order <= 1) {
        const double J = rho[2 * nx + i];
        l[d] = -a.eps * (vM[j] * J - a.xiM * J * Mj[j]);
      } else {
        l[d] = lift_value(lc, vj[j], Mj[j], rho[nx + i], rho[2 * nx + i], rho[3 * nx + i], rho[4 * nx + i],
                          rho[5 * nx + i]);
      }
    }
    gb[q] = (G)((double)gb[q] + (l[0] - l[1]));
  }
}

size_t lift_diff_ws_bytes(int nx, int batch) { return (size_t)batch * 12 * nx * sizeof(double); }

cudaError_t launch_lift_diff(const MacroArgs& a, const double* rho_new, const double* rho_old, void* g, bool fp32,
                             double* ws, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  if (fp32) lift_diff_kernel<float><<<a.batch, kMacroThreads, 0, s>>>(a, rho_new, rho_old, (float*)g, ws);
  else lift_diff_kernel<double><<<a.batch, kMacroThreads, 0, s>>>(a, rho_new, rho_old, (double*)g, ws);
  return cudaGetLastError();
}

// Sequential correction of Algorithm 1 for one solve (one CTA):
// for n = k..N-1: Gn = G(rho^{n,k+1}); rho^{n+1,k+1} = F + (Gn - Gprev);
// Gprev = Gn; err = max |rho^{n+1,k+1} - rho^{n+1,k}|.
__device__ void correct_solve(const CorrectArgs& c, const Scratch& S, double* red) {
  const MacroArgs& a = c.m;
  const int nx = a.nx;
  double emax = 0.0;
  {
    const double* rk = c.rho + (size_t)c.k * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) S.w[i] = rk[i];
    __syncthreads();
  }
  for (int n = c.k; n < c.n_slices; ++n) {
    // S.w holds rho^{n,k+1} (the previous slice's corrected density)
    coarse_block(S, a, red);
    double* out = c.rho + (size_t)(n + 1) * nx;
    const double* F = c.frho + (size_t)(n + 1) * nx;
    double* Gp = c.gprev + (size_t)(n + 1) * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double gn = S.w[i];
      const double v = F[i] + (gn - Gp[i]);
      emax = fmax(emax, fabs(v - out[i]));
      out[i] = v;
      Gp[i] = gn;
      S.w[i] = v;
    }
    __syncthreads();
  }
  for (int m = 16; m > 0; m >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, m));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double e = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) e = fmax(e, red[q]);
    *c.err = e;
  }
  __syncthreads();
}

__global__ void correct_kernel(CorrectArgs c, double* gws, int in_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  correct_solve(c, scratch_of(smem, gws, c.m.nx, in_smem), reinterpret_cast<double*>(smem));
}

// The correction of many solves, one CTA each (per-CTA scratch of `per`
// doubles when it does not fit shared memory).
__global__ void correct_list_kernel(const CorrectArgs* list, double* gws, int in_smem, size_t per) {
  extern __shared__ __align__(16) unsigned char smem[];
  const CorrectArgs& c = list[blockIdx.x];
  correct_solve(c, scratch_of(smem, gws, c.m.nx, in_smem, per), reinterpret_cast<double*>(smem));
}

// Coarse guess of Algorithm 1: rho^{n+1,0} = G(rho^{n,0}), Gprev = rho^{n+1,0}.
__device__ void coarse_chain_solve(const MacroArgs& a, int n_slices, double* rho, double* gprev, const Scratch& S,
                                   double* red) {
  const int nx = a.nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) S.w[i] = rho[i];
  __syncthreads();
  for (int n = 0; n < n_slices; ++n) {
    coarse_block(S, a, red);
    double* out = rho + (size_t)(n + 1) * nx;
    double* Gp = gprev + (size_t)(n + 1) * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      out[i] = S.w[i];
      Gp[i] = S.w[i];
    }
    __syncthreads();
  }
}

__global__ void coarse_chain_kernel(MacroArgs a, int n_slices, double* rho, double* gprev,
                                    double* gws, int in_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  coarse_chain_solve(a, n_slices, rho, gprev, scratch_of(smem, gws, a.nx, in_smem),
                     reinterpret_cast<double*>(smem));
}

// The coarse guess of many solves, one CTA each.
__global__ void coarse_chain_list_kernel(const CorrectArgs* list, double* gws, int in_smem, size_t per) {
  extern __shared__ __align__(16) unsigned char smem[];
  const CorrectArgs& c = list[blockIdx.x];
  coarse_chain_solve(c.m, c.n_slices, c.rho, c.gprev, scratch_of(smem, gws, c.m.nx, in_smem, per),
                     reinterpret_cast<double*>(smem));
}

// ------------------------------------------------------------- launches --

static size_t macro_smem(int nx, bool in_smem) {
  return 1024 + (in_smem ? 8 * ((size_t)kScratchArrays * nx + kReducedDoubles) : 0);
}
static bool macro_fits(int nx) { return macro_smem(nx, true) <= 220 * 1024; }

size_t macro_ws_bytes(int nx, int grid) {
  return macro_fits(nx) ? 0 : (size_t)grid * ((size_t)kScratchArrays * nx + kReducedDoubles) * sizeof(double);
}

// chunks of the partitioned solve: chunks of about 8 rows (the serial part of
// each thread), at most 128 (the reduced system's parallel cyclic reduction
// is then 7 levels deep), at least 4; a power of two
int coarse_parts(int nx) {
  int P = 4;
  while (P < 128 && 2 * P * 8 <= nx) P *= 2;
  return P;
}

template <class K, class... Args>
static cudaError_t launch_macro(K kernel, int grid, int nx, double* gws, cudaStream_t s,
                                Args... args) {
  const bool in_smem = macro_fits(nx);
  const size_t smem = macro_smem(nx, in_smem);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
  if (e != cudaSuccess) return e;
  if (!in_smem && gws == nullptr) return cudaErrorInvalidValue;
  kernel<<<grid, kMacroThreads, smem, s>>>(args..., gws, in_smem ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_coarse(const MacroArgs& a, const double* rho_in, double* rho_out, double* gws,
                          cudaStream_t s) {
  return launch_macro(coarse_kernel, a.batch, a.nx, gws, s, a, rho_in, rho_out);
}

cudaError_t launch_lift(const MacroArgs& a, const double* rho, void* g_out, bool fp32, double* gws,
                        cudaStream_t s) {
  if (fp32) return launch_macro(lift_kernel<float>, a.batch, a.nx, gws, s, a, rho, (float*)g_out);
  return launch_macro(lift_kernel<double>, a.batch, a.nx, gws, s, a, rho, (double*)g_out);
}

size_t macro_list_ws_bytes(int nx_max, int grid) { return macro_ws_bytes(nx_max, grid); }

static cudaError_t launch_list(void (*kernel)(const CorrectArgs*, double*, int, size_t), const CorrectArgs* list,
                               int n, int nx_max, double* gws, cudaStream_t s) {
  const bool in_smem = macro_fits(nx_max);
  const size_t smem = macro_smem(nx_max, in_smem);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
  if (e != cudaSuccess) return e;
  if (!in_smem && gws == nullptr) return cudaErrorInvalidValue;
  const size_t per = (size_t)kScratchArrays * nx_max + kReducedDoubles;
  kernel<<<n, kMacroThreads, smem, s>>>(list, gws, in_smem ? 1 : 0, per);
  return cudaGetLastError();
}

cudaError_t launch_correct_list(const CorrectArgs* list, int n, int nx_max, double* gws, cudaStream_t s) {
  return launch_list(correct_list_kernel, list, n, nx_max, gws, s);
}

cudaError_t launch_coarse_chain_list(const CorrectArgs* list, int n, int nx_max, double* gws, cudaStream_t s) {
  return launch_list(coarse_chain_list_kernel, list, n, nx_max, gws, s);
}

__global__ void __launch_bounds__(256) row_sums_kernel(const double* x, int nx, double* out) {
  __shared__ double red[8];
  const double* row = x + (size_t)blockIdx.x * nx;
  double v = 0.0;
  for (int i = threadIdx.x; i < nx; i += 256) v += row[i];
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

cudaError_t launch_row_sums(const double* x, int rows, int nx, double* out, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  row_sums_kernel<<<rows, 256, 0, s>>>(x, nx, out);
  return cudaGetLastError();
}

cudaError_t launch_correct(const CorrectArgs& c, double* gws, cudaStream_t s, bool cluster) {
  if (cluster && c.k < c.n_slices && coarse_cluster_ok(c.m)) return launch_correct_cluster(c, s);
  return launch_macro(correct_kernel, 1, c.m.nx, gws, s, c);
}

cudaError_t launch_coarse_chain(const MacroArgs& a, int n_slices, double* rho, double* gprev,
                                double* gws, cudaStream_t s, bool cluster) {
  if (cluster && n_slices > 0 && coarse_cluster_ok(a)) return launch_coarse_chain_cluster(a, n_slices, rho, gprev, s);
  return launch_macro(coarse_chain_kernel, 1, a.nx, gws, s, a, n_slices, rho, gprev);
}

}  // namespace mmk
