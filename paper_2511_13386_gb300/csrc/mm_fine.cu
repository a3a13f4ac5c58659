// Fine propagator F = S^HMM (Sec. 2.3) for a batch of slice states.
//
// One CTA of 512 threads owns one state (rho[nx], g[nx][nv]) for all the
// steps of the span, so the only synchronisation a step needs is
// __syncthreads: the Poisson law couples every cell of a state at every step
// (last line of S^MM), which rules out splitting a state across
// independently scheduled CTAs.  Per step:
//   macro phase (each thread owns a few cells): density update from the
//     interface fluxes of the previous sweep, prefix sum for E (Poisson law
//     of S^MM), the flux J of S^0, the criteria and status update of
//     Sec. 2.2-2.3 with the compaction of the interfaces to write, and the
//     per-interface constants of the sweep;
//   sweep (a group of lanes owns one interface column at a time): the g
//     update of S^MM on kinetic interfaces, g = 0 on the others, and the
//     per-lane partial velocity moments of the new g.
// g lives in two global buffers (read one, write the other each step).  A
// group walks a contiguous run of interfaces with a four-slot register ring
// holding the columns i-1, i, i+1 and the prefetch of i+2 (the loop is
// unrolled four times so the ring rotates by renaming, not by moves); each g
// value is read once and written once per step.
//
// The projection Pi = <.> M of the discrete transport needs P = <X> before
// any new g of the column can be formed.  Instead of a reduction inside the
// sweep, P is computed in the macro phase from moments of the old g:
//   <A> = ((m+_i - m+_{i-1}) - (m-_{i+1} - m-_i)) / dx,   m+- = <v^+- g>,
//   <B> = (G_{nv-3/2} - G_{1/2}) / 2   (trapezoid weights, zero end fluxes),
// which is the same sum regrouped (the x-fluxes telescope column by column,
// the v-fluxes telescope except at the two halved end weights).
//
// Precision (FP32-g path): g, the sweep and the per-lane partial moments in
// float; the density in float-float; the Poisson prefix sum in float-float;
// the per-interface moment combination by compensated (two-sum) summation;
// one float flux per interface, added to one cell and subtracted from the
// other, so mass is conserved to float-float rounding.
#include <math.h>
#include <stdio.h>

#include "ff.cuh"
#include "mm_internal.h"

namespace mmk {

// Table 1 (Sec. 2.2), offsets -3..3, rows = derivative order 1..3.
__constant__ double kFD[3][7] = {
    {-1.0 / 60, 3.0 / 20, -3.0 / 4, 0.0, 3.0 / 4, -3.0 / 20, 1.0 / 60},
    {1.0 / 90, -3.0 / 20, 3.0 / 2, -49.0 / 18, 3.0 / 2, -3.0 / 20, 1.0 / 90},
    {1.0 / 8, -1.0, 13.0 / 8, 0.0, -13.0 / 8, 1.0, -1.0 / 8}};

// ------------------------------------------------ macro-precision traits --

template <class G>
struct MP;

template <>
struct MP<double> {
  using R = double;   // density / Poisson arithmetic
  using A = double;   // moment accumulator
  static __device__ __forceinline__ R c(double x) { return x; }
  static __device__ __forceinline__ R add(R a, R b) { return a + b; }
  static __device__ __forceinline__ R sub(R a, R b) { return a - b; }
  static __device__ __forceinline__ R mul(R a, R b) { return a * b; }
  static __device__ __forceinline__ R mulg(R a, double b) { return a * b; }
  static __device__ __forceinline__ R addg(R a, double b) { return a + b; }
  static __device__ __forceinline__ double tod(R a) { return a; }
  static __device__ __forceinline__ double tog(R a) { return a; }
  static __device__ __forceinline__ R zero() { return 0.0; }
  static __device__ __forceinline__ R shfl_up(R a, int d) { return __shfl_up_sync(0xffffffffu, a, d); }
  static __device__ __forceinline__ R shfl_xor(R a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
  // moments
  static __device__ __forceinline__ A azero() { return 0.0; }
  static __device__ __forceinline__ A aadd(A s, double x) { return s + x; }
  static __device__ __forceinline__ double aval(A s, double k) { return s * k; }
  // J from two densities and E
  static __device__ __forceinline__ double flux_J(R r0, R r1, double e, double inv_dx) {
    return (r1 - r0) * inv_dx - e * 0.5 * (r0 + r1);
  }
};

template <>
struct MP<float> {
  using R = ff;
  struct A {
    float s, e;
  };
  static __device__ __forceinline__ R c(double x) { return ff_from_double(x); }
  static __device__ __forceinline__ R add(R a, R b) { return ff_add(a, b); }
  static __device__ __forceinline__ R sub(R a, R b) { return ff_sub(a, b); }
  static __device__ __forceinline__ R mul(R a, R b) { return ff_mul(a, b); }
  static __device__ __forceinline__ R mulg(R a, float b) { return ff_mul_f(a, b); }
  static __device__ __forceinline__ R addg(R a, float b) { return ff_add_f(a, b); }
  static __device__ __forceinline__ double tod(R a) { return ff_to_double(a); }
  static __device__ __forceinline__ float tog(R a) { return a.hi; }
  static __device__ __forceinline__ R zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ R shfl_up(R a, int d) { return ff_shfl_up(a, d); }
  static __device__ __forceinline__ R shfl_xor(R a, int m) { return ff_shfl_xor(a, m); }
  // compensated (two-sum) accumulation of float terms
  static __device__ __forceinline__ A azero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ A aadd(A a, float x) {
    const ff t = two_sum(a.s, x);
    return {t.hi, __fadd_rn(a.e, t.lo)};
  }
  static __device__ __forceinline__ float aval(A a, float k) { return __fmaf_rn(a.s, k, __fmul_rn(a.e, k)); }
  static __device__ __forceinline__ float flux_J(R r0, R r1, float e, float inv_dx) {
    const float dr = ff_sub(r1, r0).hi;
    return dr * inv_dx - e * 0.5f * (r0.hi + r1.hi);
  }
};

// ------------------------------------------------------- column arrays ---

// Offsets of the per-state column arrays; identical on host and device.
struct ColLayout {
  size_t rho, S, jg, mp, mm, part, n2, ends, par, list, ed, rd, jd, cell0, cell1, kin0, kin1, kin2, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline ColLayout col_layout(int nx, int lanes, int gbytes, bool adapt) {
  ColLayout L;
  const size_t n = nx;
  size_t o = 0;
  L.rho = o;  o = al16(o + 8 * n);
  L.S = o;    o = al16(o + 8 * n);
  L.jg = o;   o = al16(o + gbytes * n);
  L.mp = o;   o = al16(o + gbytes * n);
  L.mm = o;   o = al16(o + gbytes * n);
  L.part = o; o = al16(o + gbytes * n * lanes);
  L.ends = o; o = al16(o + gbytes * n * 4);
  L.par = o;  o = al16(o + gbytes * n * 4);
  L.n2 = o;   if (adapt) o = al16(o + gbytes * n * lanes);
  L.list = o; if (adapt) o = al16(o + 4 * n);
  L.ed = o;   if (adapt) o = al16(o + 8 * n);
  L.rd = o;   if (adapt) o = al16(o + 8 * n);
  L.jd = o;   if (adapt) o = al16(o + 8 * n);
  L.cell0 = o; if (adapt) o = al16(o + n);
  L.cell1 = o; if (adapt) o = al16(o + n);
  L.kin0 = o;  if (adapt) o = al16(o + n);
  L.kin1 = o;  if (adapt) o = al16(o + n);
  L.kin2 = o;  if (adapt) o = al16(o + n);
  L.total = o;
  return L;
}

constexpr int kRedSlots = 160;  // reduction scratch entries (8 bytes each)

size_t fine_column_bytes(int nx, int nv, int lanes, bool fp32, bool adapt) {
  (void)nv;
  return col_layout(nx, lanes, fp32 ? 4 : 8, adapt).total;
}

size_t fine_smem_bytes(int nx, int nv, int lanes, bool fp32, bool adapt, bool col_in_smem) {
  size_t s = 8 * (size_t)kRedSlots;
  if (col_in_smem) s += fine_column_bytes(nx, nv, lanes, fp32, adapt);
  return s;
}

// -------------------------------------------------------- vector access ---

template <class G, int V>
__device__ __forceinline__ void vload(G (&r)[V], const G* p) {
  constexpr int B = V * (int)sizeof(G);
  if constexpr (B % 16 == 0) {
#pragma unroll
    for (int q = 0; q < B / 16; ++q) {
      const float4 t = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(p) + 16 * q);
      const G* tg = reinterpret_cast<const G*>(&t);
#pragma unroll
      for (int e = 0; e < 16 / (int)sizeof(G); ++e) r[q * (16 / sizeof(G)) + e] = tg[e];
    }
  } else if constexpr (B % 8 == 0) {
#pragma unroll
    for (int q = 0; q < B / 8; ++q) {
      const float2 t = *reinterpret_cast<const float2*>(reinterpret_cast<const char*>(p) + 8 * q);
      const G* tg = reinterpret_cast<const G*>(&t);
#pragma unroll
      for (int e = 0; e < 8 / (int)sizeof(G); ++e) r[q * (8 / sizeof(G)) + e] = tg[e];
    }
  } else {
#pragma unroll
    for (int e = 0; e < V; ++e) r[e] = p[e];
  }
}

template <class G, int V>
__device__ __forceinline__ void vstore(G* p, const G (&r)[V]) {
  constexpr int B = V * (int)sizeof(G);
  if constexpr (B % 16 == 0) {
#pragma unroll
    for (int q = 0; q < B / 16; ++q) {
      float4 t;
      G* tg = reinterpret_cast<G*>(&t);
#pragma unroll
      for (int e = 0; e < 16 / (int)sizeof(G); ++e) tg[e] = r[q * (16 / sizeof(G)) + e];
      *reinterpret_cast<float4*>(reinterpret_cast<char*>(p) + 16 * q) = t;
    }
  } else if constexpr (B % 8 == 0) {
#pragma unroll
    for (int q = 0; q < B / 8; ++q) {
      float2 t;
      G* tg = reinterpret_cast<G*>(&t);
#pragma unroll
      for (int e = 0; e < 8 / (int)sizeof(G); ++e) tg[e] = r[q * (8 / sizeof(G)) + e];
      *reinterpret_cast<float2*>(reinterpret_cast<char*>(p) + 8 * q) = t;
    }
  } else {
#pragma unroll
    for (int e = 0; e < V; ++e) p[e] = r[e];
  }
}

// ----------------------------------------------------- block reductions --

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
  __syncthreads();
  return t;
}

// Exclusive block scan of ints a (returned) with block totals of a and b.
__device__ __forceinline__ int block_scan2_i(int a, int b, int* red, int* tot_a, int* tot_b) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  int inc = a;
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, d);
    if (l >= d) inc += t;
  }
  int bs = b;
  for (int m = 16; m > 0; m >>= 1) bs += __shfl_xor_sync(0xffffffffu, bs, m);
  __syncthreads();
  if (l == 31) red[w] = inc;
  if (l == 0) red[32 + w] = bs;
  __syncthreads();
  int off = 0, ta = 0, tb = 0;
  const int nw = blockDim.x >> 5;
  for (int q = 0; q < nw; ++q) {
    if (q < w) off += red[q];
    ta += red[q];
    tb += red[32 + q];
  }
  __syncthreads();
  *tot_a = ta;
  *tot_b = tb;
  return off + inc - a;
}

// ------------------------------------------------------------ the kernel --

template <class G>
struct Cols {
  using R = typename MP<G>::R;
  R *rho, *S;
  G *jg, *mp, *mm, *part, *n2, *ends, *par;
  int* list;
  double *ed, *rd, *jd;
  uint8_t *cell0, *cell1, *kin0, *kin1, *kin2;
};

template <class G>
__device__ __forceinline__ Cols<G> carve(unsigned char* base, int nx, int lanes, bool adapt) {
  using R = typename MP<G>::R;
  const ColLayout L = col_layout(nx, lanes, sizeof(G), adapt);
  Cols<G> c;
  c.rho = reinterpret_cast<R*>(base + L.rho);
  c.S = reinterpret_cast<R*>(base + L.S);
  c.jg = reinterpret_cast<G*>(base + L.jg);
  c.mp = reinterpret_cast<G*>(base + L.mp);
  c.mm = reinterpret_cast<G*>(base + L.mm);
  c.part = reinterpret_cast<G*>(base + L.part);
  c.n2 = reinterpret_cast<G*>(base + L.n2);
  c.ends = reinterpret_cast<G*>(base + L.ends);
  c.par = reinterpret_cast<G*>(base + L.par);
  c.list = reinterpret_cast<int*>(base + L.list);
  c.ed = reinterpret_cast<double*>(base + L.ed);
  c.rd = reinterpret_cast<double*>(base + L.rd);
  c.jd = reinterpret_cast<double*>(base + L.jd);
  c.cell0 = base + L.cell0;
  c.cell1 = base + L.cell1;
  c.kin0 = base + L.kin0;
  c.kin1 = base + L.kin1;
  c.kin2 = base + L.kin2;
  return c;
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Lifting of order one (Def. 1, identification l = 0 of Sec. 2.1) of one
// density into g, by the whole block, in double: the Poisson law of S^MM
// (prefix sum, mean-zero gauge), J of S^0, then
// g_{i+1/2,j} = -eps (xi_j M_j - <xi M> M_j) J_{i+1/2}.  E and J use the
// first 16 nx bytes of `scratch`.
template <class G>
__device__ void lift_block(const FineArgs& A, const double* rho, double rb, G* g, unsigned char* scratch,
                           double* red) {
  const int nx = A.nx, nv = A.nv, T = blockDim.x, tid = threadIdx.x;
  double* E = reinterpret_cast<double*>(scratch);
  double* J = E + nx;
  const int cpt = (nx + T - 1) / T;
  const int c0 = min(tid * cpt, nx), c1 = min(c0 + cpt, nx);
  double t1 = 0.0, t2 = 0.0;
  for (int c = c0; c < c1; ++c) {
    const double d = (rho[c] - rb) * A.dx;
    t1 += d;
    E[c] = t1;
    t2 += d * (double)(nx - c);
  }
  const int w = tid >> 5, l = tid & 31, nw = T >> 5;
  double inc = t1;
  for (int d = 1; d < 32; d <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, inc, d);
    if (l >= d) inc += t;
  }
  double ex = __shfl_up_sync(0xffffffffu, inc, 1);
  if (l == 0) ex = 0.0;
  for (int m = 16; m > 0; m >>= 1) t2 += __shfl_xor_sync(0xffffffffu, t2, m);
  __syncthreads();
  if (l == 31) red[w] = inc;
  if (l == 0) red[32 + w] = t2;
  __syncthreads();
  double off = 0.0, tw = 0.0;
  for (int q = 0; q < nw; ++q) {
    if (q < w) off += red[q];
    tw += red[32 + q];
  }
  const double mean = tw * (1.0 / nx), base = off + ex;
  for (int c = c0; c < c1; ++c) E[c] = base + E[c] - mean;
  __syncthreads();
  for (int c = c0; c < c1; ++c) {
    const double r0 = rho[c], r1 = rho[c + 1 == nx ? 0 : c + 1];
    J[c] = (r1 - r0) * A.inv_dx - E[c] * 0.5 * (r0 + r1);
  }
  __syncthreads();
  const double* vM = A.vtab + 2 * nv;
  const double* Mj = A.vtab + 1 * nv;
  const unsigned n = (unsigned)nx * (unsigned)nv;
  for (unsigned q = tid; q < n; q += T) {
    const unsigned i = q / (unsigned)nv, j = q - i * (unsigned)nv;
    const double Ji = J[i];
    g[q] = (G)(-A.eps * (vM[j] * Ji - A.xiM * Ji * Mj[j]));
  }
  __syncthreads();
}

// F for one state: n_steps steps from (rin, gin); gin == nullptr lifts the
// density first.  buf0/buf1 are the two step buffers (the last step writes
// buf0); colbase holds the column arrays (shared or global memory).
template <class G, int VPT, bool ADAPT, bool CSMEM>
__device__ __forceinline__ void fine_state(const FineArgs& A, const double* rin, const G* gin, G* buf0, G* buf1,
                                           double* rout, uint8_t* mout, unsigned char* smem,
                                           unsigned char* colbase) {
  using M = MP<G>;
  using R = typename M::R;
  using Acc = typename M::A;

  const int tid = threadIdx.x;
  const int nx = A.nx, nv = A.nv, Lg = A.lanes;
  constexpr int T = kFineThreads;

  double* red = reinterpret_cast<double*>(smem);
  if (gin == nullptr) {  // the lifted density goes where the first step does not write
    G* lifted = (A.n_steps & 1) ? buf1 : buf0;
    lift_block<G>(A, rin, A.rho_bar, lifted, colbase, red);
    gin = lifted;
  }
  Cols<G> C = carve<G>(colbase, nx, Lg, ADAPT);

  // ---- ownership of cells in the macro phase
  const int cpt = (nx + T - 1) / T;
  const int c0 = min(tid * cpt, nx), c1 = min(c0 + cpt, nx);

  // ---- lane layout of the sweep
  const int lig = tid % Lg;                // lane in group
  const int grp = tid / Lg;
  const int ngrp = T / Lg;
  const bool pos = lig >= A.nhp;
  const int hl = pos ? lig - A.nhp : lig;  // lane within its half
  const bool active = hl < A.nh;
  const int j0 = pos ? nv / 2 + hl * VPT : hl * VPT;
  const bool first_lane = active && j0 == 0;
  const bool last_lane = active && j0 + VPT == nv;
  const int warp_base = (tid & 31) - lig;  // first lane of this group in the warp
  const int src_left = warp_base + ((lig == A.nhp) ? A.nh - 1 : max(lig - 1, 0));
  const int src_right = warp_base + ((lig == A.nh - 1) ? A.nhp : min(lig + 1, Lg - 1));
  // which of the four end values (g_0, g_1, g_{nv-2}, g_{nv-1}) this lane stores
  int end_slot = -1;
  if (VPT == 1 && active) end_slot = j0 == 0 ? 0 : j0 == 1 ? 1 : j0 == nv - 2 ? 2 : j0 == nv - 1 ? 3 : -1;

  // per-node constants of this lane: |v|/dx, M, v M, w v, w
  G av[VPT], Mj[VPT], xM[VPT], wv[VPT], wj[ADAPT ? VPT : 1];
  {
    const G* tab = sizeof(G) == 4 ? reinterpret_cast<const G*>(A.vtab_f) : reinterpret_cast<const G*>(A.vtab);
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const int j = active ? j0 + k : 0;
      av[k] = active ? tab[0 * nv + j] : G(0);
      Mj[k] = active ? tab[1 * nv + j] : G(0);
      xM[k] = active ? tab[2 * nv + j] : G(0);
      wv[k] = active ? tab[3 * nv + j] : G(0);
      if constexpr (ADAPT) wj[k] = active ? tab[4 * nv + j] : G(0);
    }
  }
  // scalar constants in the working precisions (converted once)
  const G ga = (G)A.a, gb = (G)A.b, g_inv_dx = (G)A.inv_dx, g_inv_dv = (G)A.inv_dv;
  const G g_kflux = (G)(A.dt_dx * A.inv_eps);    // dt/dx <xi g> / eps
  const G g_fflux = (G)(-A.dt_dx * A.m2);        // dt/dx (-m2 J)
  const R Rdx = M::c(A.dx), Rinv_nx = M::c(1.0 / nx);

  // ---- prologue: density, rho_bar, moments of g_in
  double rb = A.rho_bar;
  {
    double s = 0.0;
    for (int c = c0; c < c1; ++c) {
      const double r = rin[c];
      C.rho[c] = M::c(r);
      s += r;
    }
    if (isnan(rb)) rb = block_sum_d(s, red) / nx;
  }
  const R Rrb = M::c(rb);

  for (int i = grp; i < nx; i += ngrp) {
    G w1[VPT];
#pragma unroll
    for (int k = 0; k < VPT; ++k) w1[k] = G(0);
    if (active) vload<G, VPT>(w1, gin + (size_t)i * nv + j0);
    G p = 0, q = 0;
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      p += wv[k] * w1[k];
      if constexpr (ADAPT) q += wj[k] * w1[k] * w1[k];
    }
    C.part[(size_t)i * Lg + lig] = p;
    if constexpr (ADAPT) C.n2[(size_t)i * Lg + lig] = q;
    if constexpr (VPT >= 2) {
      if (first_lane) { C.ends[4 * i + 0] = w1[0]; C.ends[4 * i + 1] = w1[1]; }
      if (last_lane) { C.ends[4 * i + 2] = w1[VPT - 2]; C.ends[4 * i + 3] = w1[VPT - 1]; }
    } else {
      if (end_slot >= 0) C.ends[4 * i + end_slot] = w1[0];
    }
  }
  if constexpr (ADAPT) {
    for (int c = c0; c < c1; ++c) { C.kin1[c] = 1; C.kin2[c] = 1; }
  }
  __syncthreads();

  // moments m+- of the current g from the lane partials (own cells)
  auto moments = [&](int c) {
    G sp = 0, sm = 0;
    const G* pp = C.part + c * Lg;
    for (int l = 0; l < Lg; ++l) {
      if (l >= A.nhp) sp += pp[l];
      else sm += pp[l];
    }
    C.mp[c] = sp;
    C.mm[c] = -sm;
  };
  for (int c = c0; c < c1; ++c) moments(c);

  uint8_t* cell_cur = C.cell0;   // s^n
  uint8_t* cell_nxt = C.cell1;   // s^{n+1}
  uint8_t* kin_cur = C.kin0;     // interface flags under s^n
  uint8_t* kin_prev = C.kin1;    // under s^{n-1}
  uint8_t* kin_prev2 = C.kin2;   // under s^{n-2}
  int* ired = reinterpret_cast<int*>(red);
  int count = nx;                // interfaces to write this step
  long long kin_total = 0;       // kinetic interfaces summed over steps (thread 0)
  const int w = tid >> 5, l = tid & 31;

  // ------------------------------------------------------------ macro A --
  // E, J, criteria/status, write list and sweep constants for step n.
  auto macro_A = [&](bool initial) {
    // Poisson law: S_c = sum_{m<=c} (rho_m - rho_bar) dx ; E = S - mean(S),
    // with mean(S) = sum_m (nx - m) d_m / nx.
    R t1 = M::zero(), t2 = M::zero();
    G wgt = G(nx - c0);  // nx - c, counted down without an int conversion
    for (int c = c0; c < c1; ++c) {
      const R d = M::mul(M::sub(C.rho[c], Rrb), Rdx);
      t1 = M::add(t1, d);
      C.S[c] = t1;
      t2 = M::add(t2, M::mulg(d, wgt));
      wgt -= G(1);
    }
    R inc = t1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const R t = M::shfl_up(inc, d);
      if (l >= d) inc = M::add(inc, t);
    }
    R ex_lane = M::shfl_up(inc, 1);
    if (l == 0) ex_lane = M::zero();
    R ws = t2;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) ws = M::add(ws, M::shfl_xor(ws, m));
    R* rr = reinterpret_cast<R*>(red);
    if (l == 31) rr[w] = inc;
    if (l == 0) rr[32 + w] = ws;
    __syncthreads();
    if (w == 0) {  // exclusive scan of the warp totals and the mean, once
      constexpr int NW = T / 32;
      R v = l < NW ? rr[l] : M::zero();
      R u = l < NW ? rr[32 + l] : M::zero();
#pragma unroll
      for (int d = 1; d < NW; d <<= 1) {
        const R t = M::shfl_up(v, d);
        if (l >= d) v = M::add(v, t);
      }
#pragma unroll
      for (int m = NW / 2; m > 0; m >>= 1) u = M::add(u, M::shfl_xor(u, m));
      R ex = M::shfl_up(v, 1);
      if (l == 0) ex = M::zero();
      if (l < NW) rr[64 + l] = ex;
      if (l == 0) rr[96] = M::mul(u, Rinv_nx);
    }
    __syncthreads();
    const R base = M::add(rr[64 + w], ex_lane);
    const R meanS = rr[96];
    G* eg = C.par;  // E^n goes through the par array's first slot first
    for (int c = c0; c < c1; ++c) {
      const R E = M::sub(M::add(base, C.S[c]), meanS);
      eg[4 * c + 3] = (G)M::tog(E);          // temporary: E in slot 3
      if constexpr (ADAPT) { C.ed[c] = M::tod(E); C.rd[c] = M::tod(C.rho[c]); }
    }
    __syncthreads();  // rho final for this step; E of all cells visible

    if constexpr (ADAPT) {
      // criteria of Sec. 2.2 in double: remainder R (eq. Remainder with
      // Table 1), interface norms ||g||_2; status update of Sec. 2.3.
      const double inv_dx = A.inv_dx;
      auto rho_d = [&](int c) { return C.rd[wrapi(c, nx)]; };
      auto E_d = [&](int c) { return C.ed[wrapi(c, nx)]; };
      double jsum = 0.0;
      for (int c = c0; c < c1; ++c) {
        double d1 = 0.0;
        for (int k = -3; k <= 3; ++k) d1 += kFD[0][k + 3] * rho_d(c + k);
        d1 *= inv_dx;
        const double Ec = 0.5 * (E_d(c - 1) + E_d(c));
        C.jd[c] = d1 - Ec * rho_d(c);
        jsum += C.jd[c];
      }
      const double meanJ = block_sum_d(jsum, red) / nx;  // (syncs: Jc visible)
      const double r2 = 1.0 / (A.dx * A.dx), r3 = r2 / A.dx;
      for (int c = c0; c < c1; ++c) {
        double d1r = 0.0, d1J = 0.0, d2J = 0.0, d3J = 0.0;
        for (int k = -3; k <= 3; ++k) {
          const double jk = C.jd[wrapi(c + k, nx)];
          d1r += kFD[0][k + 3] * rho_d(c + k);
          d1J += kFD[0][k + 3] * jk;
          d2J += kFD[1][k + 3] * jk;
          d3J += kFD[2][k + 3] * jk;
        }
        d1r *= inv_dx; d1J *= inv_dx; d2J *= r2; d3J *= r3;
        const double Ec = 0.5 * (E_d(c - 1) + E_d(c));
        const double rc = rho_d(c);
        const double Rc = -d3J + Ec * d2J + (2.0 * rc - 3.0 * rb) * d1J + 2.0 * C.jd[c] * d1r -
                          d1r * (C.jd[c] - meanJ);
        const bool big_R = A.r_fac * fabs(Rc) > A.thr_R;
        double nl = 0.0, nr = 0.0;
        const G* pl = C.n2 + wrapi(c - 1, nx) * Lg;
        const G* pr = C.n2 + c * Lg;
        for (int q = 0; q < Lg; ++q) { nl += (double)pl[q]; nr += (double)pr[q]; }
        nl = sqrt(nl); nr = sqrt(nr);
        uint8_t s;
        if (initial) {
          s = (nl > A.thr_g || nr > A.thr_g || big_R) ? 1 : 0;
          cell_cur[c] = s;
        }
        const uint8_t cur = initial ? s : cell_cur[c];
        if (!cur) s = big_R ? 1 : 0;
        else s = (nl <= A.thr_g && nr <= A.thr_g && !big_R) ? 0 : 1;
        cell_nxt[c] = s;
      }
      __syncthreads();  // cell_cur of all cells visible

      // interface flags under s^n; an interface is written while it is
      // kinetic and for the two steps after it turns fluid, so that both
      // step buffers hold its zeros
      int nw = 0, nk = 0;
      for (int c = c0; c < c1; ++c) {
        const uint8_t k = cell_cur[c] | cell_cur[wrapi(c + 1, nx)];
        kin_cur[c] = k;
        nk += k;
        nw += (k | kin_prev[c] | kin_prev2[c]) ? 1 : 0;
      }
      int tot_w, tot_k;
      int pos0 = block_scan2_i(nw, nk, ired, &tot_w, &tot_k);
      for (int c = c0; c < c1; ++c)
        if (kin_cur[c] | kin_prev[c] | kin_prev2[c]) C.list[pos0++] = c;
      count = tot_w;
      if (tid == 0) kin_total += tot_k;
    } else {
      count = nx;
      if (tid == 0) kin_total += nx;
    }

    // J and the sweep constants: E+/dv, E-/dv, P = <X>, J
    for (int c = c0; c < c1; ++c) {
      const int cl = wrapi(c - 1, nx), cr = wrapi(c + 1, nx);
      G* pr = C.par + 4 * c;
      const G e = pr[3];
      const G J = M::flux_J(C.rho[c], C.rho[cr], e, g_inv_dx);
      C.jg[c] = J;
      const G ep = e > G(0) ? e : G(0), em = e < G(0) ? -e : G(0);
      const G pm = ((C.mp[c] - C.mp[cl]) - (C.mm[cr] - C.mm[c])) * g_inv_dx;
      const G* en = C.ends + 4 * c;
      const G gend = (G)0.5 * ((ep * en[2] - em * en[3]) - (ep * en[0] - em * en[1]));
      pr[0] = ep * g_inv_dv;
      pr[1] = em * g_inv_dv;
      pr[2] = pm + gend;
      pr[3] = J;
    }
    __syncthreads();
  };

  // ------------------------------------------------------------ macro C --
  // density update from the fluxes of the new g: one flux per interface
  // (kinetic: dt/dx <xi g>/eps, fluid: dt/dx (-m2 J)), or the cell-based
  // rule of S^HMM when flux_rule == 1.
  auto flux_kin = [&](int c) {
    Acc s = M::azero();
    const G* pp = C.part + c * Lg;
    for (int q = 0; q < Lg; ++q) s = M::aadd(s, pp[q]);
    return (G)M::aval(s, g_kflux);
  };
  auto is_kin = [&](int c) { return ADAPT ? kin_cur[c] != 0 : true; };
  auto macro_C = [&]() {
    if (c0 < c1) {
      if (A.flux_rule == 0) {
        const int cl = wrapi(c0 - 1, nx);
        G Fp = is_kin(cl) ? flux_kin(cl) : g_fflux * C.jg[cl];
        for (int c = c0; c < c1; ++c) {
          const G Fc = is_kin(c) ? flux_kin(c) : g_fflux * C.jg[c];
          C.rho[c] = M::addg(M::addg(C.rho[c], Fp), -Fc);
          Fp = Fc;
        }
      } else {
        for (int c = c0; c < c1; ++c) {
          const int cl = wrapi(c - 1, nx);
          G Fr, Fl;
          if (!ADAPT || cell_cur[c]) {
            Fr = is_kin(c) ? flux_kin(c) : G(0);
            Fl = is_kin(cl) ? flux_kin(cl) : G(0);
          } else {
            Fr = g_fflux * C.jg[c];
            Fl = g_fflux * C.jg[cl];
          }
          C.rho[c] = M::addg(M::addg(C.rho[c], Fl), -Fr);
        }
      }
    }
    for (int c = c0; c < c1; ++c) moments(c);
  };

  // --------------------------------------------------------------- sweep --

  auto sweep = [&](const G* src, G* dst) {
    const int epg = (count + ngrp - 1) / ngrp;
    const int e0 = grp * epg, e1 = min(e0 + epg, count);
    G R0[VPT], R1[VPT], R2[VPT], R3[VPT];
#pragma unroll
    for (int k = 0; k < VPT; ++k) R0[k] = R1[k] = R2[k] = R3[k] = G(0);
    int last = -10;
    auto col = [&](int i) { return src + (unsigned)(wrapi(i, nx) * nv + j0); };
    // one interface column: P = g(i-1), Cc = g(i), N = g(i+1), F = g(i+2)
    // (in flight); afterwards P receives g(i+3).
    auto body = [&](int e, G(&P)[VPT], G(&Cc)[VPT], G(&N)[VPT], G(&F)[VPT]) {
      const bool valid = e < e1;
      const int i = valid ? (ADAPT ? C.list[e] : e) : last + 1;
      if (valid && i != last + 1 && active) {
        vload<G, VPT>(P, col(i - 1));
        vload<G, VPT>(Cc, col(i));
        vload<G, VPT>(N, col(i + 1));
        vload<G, VPT>(F, col(i + 2));
      }
      last = i;
      const G left_nb = __shfl_sync(0xffffffffu, Cc[VPT - 1], src_left);
      const G right_nb = __shfl_sync(0xffffffffu, Cc[0], src_right);
      if (valid) {
        const bool kin = ADAPT ? (kin_cur[i] != 0) : true;
        G out[VPT];
        G psum = 0, nsum = 0;
        if (kin) {
          const float4* pr4 = reinterpret_cast<const float4*>(C.par + 4 * i);
          G Ep, Em, Pp, Jv;
          if constexpr (sizeof(G) == 4) {
            const float4 q = *pr4;
            Ep = q.x; Em = q.y; Pp = q.z; Jv = q.w;
          } else {
            const G* pr = C.par + 4 * i;
            Ep = pr[0]; Em = pr[1]; Pp = pr[2]; Jv = pr[3];
          }
          G Gl = first_lane ? G(0) : (Ep * left_nb - Em * Cc[0]);
#pragma unroll
          for (int k = 0; k < VPT; ++k) {
            const G c = Cc[k];
            const G u = pos ? P[k] : N[k];
            const G Ax = av[k] * (c - u);
            const G cr = (k < VPT - 1) ? Cc[(k + 1 < VPT) ? k + 1 : k] : right_nb;
            G Gr = Ep * c - Em * cr;
            if (k == VPT - 1 && last_lane) Gr = G(0);
            const G X = Ax + (Gr - Gl);
            Gl = Gr;
            const G inner = X - Pp * Mj[k] + Jv * xM[k];
            const G gs = ga * c - gb * inner;
            out[k] = gs;
            psum += wv[k] * gs;
            if constexpr (ADAPT) nsum += wj[k] * gs * gs;
          }
        } else {
#pragma unroll
          for (int k = 0; k < VPT; ++k) out[k] = G(0);
        }
        if (active) {
          vstore<G, VPT>(dst + (unsigned)(i * nv + j0), out);
          if (valid) vload<G, VPT>(P, col(i + 3));
        }
        C.part[i * Lg + lig] = psum;
        if constexpr (ADAPT) C.n2[i * Lg + lig] = nsum;
        if constexpr (VPT >= 2) {
          if (first_lane) { C.ends[4 * i + 0] = out[0]; C.ends[4 * i + 1] = out[1]; }
          if (last_lane) { C.ends[4 * i + 2] = out[VPT - 2]; C.ends[4 * i + 3] = out[VPT - 1]; }
        } else {
          if (end_slot >= 0) C.ends[4 * i + end_slot] = out[0];
        }
      }
    };
    for (int e = e0; e < e0 + epg; e += 4) {
      body(e + 0, R0, R1, R2, R3);
      body(e + 1, R1, R2, R3, R0);
      body(e + 2, R2, R3, R0, R1);
      body(e + 3, R3, R0, R1, R2);
    }
  };

  // ------------------------------------------------------------ step loop --
  macro_A(true);
  const G* src = gin;
  for (int64_t s = 0; s < A.n_steps; ++s) {
    G* dst = ((A.n_steps - 1 - s) & 1) ? buf1 : buf0;
    sweep(src, dst);
    __syncthreads();
    macro_C();
    if constexpr (ADAPT) {  // s^{n+1} becomes current; flag history shifts
      uint8_t* t = cell_cur; cell_cur = cell_nxt; cell_nxt = t;
      t = kin_prev2; kin_prev2 = kin_prev; kin_prev = kin_cur; kin_cur = t;
    }
    if (s + 1 < A.n_steps) macro_A(false);
    src = dst;
  }
  __syncthreads();

  // ---- epilogue
  int bad = 0;
  for (int c = c0; c < c1; ++c) {
    const double r = M::tod(C.rho[c]);
    rout[c] = r;
    if (!isfinite(r)) bad = 1;
    if (mout) mout[c] = ADAPT ? cell_cur[c] : 1;
  }
  if (bad) atomicExch(A.status, (int)MM_ERR_UNSTABLE);
  if (tid == 0 && A.kin_count) atomicAdd(A.kin_count, (unsigned long long)kin_total * (unsigned long long)nv);
}

// One CTA per state of a uniform batch.
template <class G, int VPT, bool ADAPT, bool CSMEM>
__global__ void __launch_bounds__(kFineThreads, 1) fine_kernel(const FineArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t st = blockIdx.x;
  const size_t sz = (size_t)A.nx * A.nv;
  unsigned char* colbase = CSMEM ? smem + 8 * kRedSlots
                                 : reinterpret_cast<unsigned char*>(A.col_ws) + st * A.col_ws_stride;
  fine_state<G, VPT, ADAPT, CSMEM>(A, A.rho_in + st * A.nx, reinterpret_cast<const G*>(A.g_in) + st * sz,
                                   reinterpret_cast<G*>(A.g_buf0) + st * sz,
                                   reinterpret_cast<G*>(A.g_buf1) + st * sz, A.rho_out + st * A.nx,
                                   A.mask_out ? A.mask_out + st * A.nx : nullptr, smem, colbase);
}

// Persistent work-list kernel: each CTA takes (solve, slice) items from a
// global counter until the list is exhausted (dynamic scheduling of uneven
// fine propagations; the list is sorted by decreasing cost on the host).
// An item propagates rho^{n,k} of its solve (g from slice 0's data, or
// lifted from the density) and writes F(rho)^{n+1}.  The step buffers and
// (when they do not fit shared memory) the column arrays are per-CTA
// workspace reused from item to item.
template <class G, int VPT, bool ADAPT, bool CSMEM>
__global__ void __launch_bounds__(kFineThreads, 1)
    fine_list_kernel(const FineListSolve* solves, const FineListItem* items, int n_items, int* next,
                     unsigned char* ws, size_t ws_g, size_t ws_col) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ __align__(16) FineArgs s_args;
  unsigned char* mine = ws + (size_t)blockIdx.x * (2 * ws_g + (CSMEM ? 0 : ws_col));
  G* b0 = reinterpret_cast<G*>(mine);
  G* b1 = reinterpret_cast<G*>(mine + ws_g);
  unsigned char* colbase = CSMEM ? smem + 8 * kRedSlots : mine + 2 * ws_g;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int k = s_item;
    if (k >= n_items) break;
    const FineListItem it = items[k];
    const FineListSolve* S = solves + it.solve;
    {  // the solve's arguments into shared memory (broadcast reads)
      const int* src = reinterpret_cast<const int*>(&S->a);
      int* dst = reinterpret_cast<int*>(&s_args);
      for (int q = threadIdx.x; q < (int)(sizeof(FineArgs) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    const int nx = s_args.nx;
    const G* gin = (it.slice == 0 && S->g0) ? reinterpret_cast<const G*>(S->g0) : nullptr;
    fine_state<G, VPT, ADAPT, CSMEM>(s_args, S->rho + (size_t)it.slice * nx, gin, b0, b1,
                                     S->frho + (size_t)(it.slice + 1) * nx, nullptr, smem, colbase);
    __syncthreads();  // before the next item overwrites s_args, s_item and the buffers
  }
}

// ---------------------------------------------------------------- launch --

template <class G, int VPT, bool ADAPT, bool CSMEM>
static cudaError_t launch_t(const FineArgs& a, size_t smem, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(fine_kernel<G, VPT, ADAPT, CSMEM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  fine_kernel<G, VPT, ADAPT, CSMEM><<<a.batch, kFineThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <class G, int VPT>
static cudaError_t launch_v(const FineArgs& a, size_t smem, cudaStream_t s) {
  if (a.adapt) {
    return a.col_in_smem ? launch_t<G, VPT, true, true>(a, smem, s) : launch_t<G, VPT, true, false>(a, smem, s);
  }
  return a.col_in_smem ? launch_t<G, VPT, false, true>(a, smem, s) : launch_t<G, VPT, false, false>(a, smem, s);
}

template <class G, int VPT, bool ADAPT, bool CSMEM>
static cudaError_t launch_list_t(const FineList& L, size_t smem, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(fine_list_kernel<G, VPT, ADAPT, CSMEM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  fine_list_kernel<G, VPT, ADAPT, CSMEM><<<L.grid, kFineThreads, smem, s>>>(L.solves, L.items, L.n_items, L.next,
                                                                            L.ws, L.ws_g, L.ws_col);
  return cudaGetLastError();
}

cudaError_t launch_fine_list(const FineList& L, bool fp32, bool adapt, bool col_in_smem, size_t smem,
                             cudaStream_t s) {
  if (fp32) {
    if (adapt) return col_in_smem ? launch_list_t<float, 8, true, true>(L, smem, s)
                                  : launch_list_t<float, 8, true, false>(L, smem, s);
    return col_in_smem ? launch_list_t<float, 8, false, true>(L, smem, s)
                       : launch_list_t<float, 8, false, false>(L, smem, s);
  }
  if (adapt) return col_in_smem ? launch_list_t<double, 4, true, true>(L, smem, s)
                                : launch_list_t<double, 4, true, false>(L, smem, s);
  return col_in_smem ? launch_list_t<double, 4, false, true>(L, smem, s)
                     : launch_list_t<double, 4, false, false>(L, smem, s);
}

cudaError_t launch_fine(const FineArgs& args, int vpt, bool fp32, size_t smem, cudaStream_t s) {
  FineArgs a = args;
  fine_args_floats(a);
  if (fp32) {
    switch (vpt) {
      case 1: return launch_v<float, 1>(a, smem, s);
      case 2: return launch_v<float, 2>(a, smem, s);
      case 4: return launch_v<float, 4>(a, smem, s);
      case 8: return launch_v<float, 8>(a, smem, s);
    }
  } else {
    switch (vpt) {
      case 1: return launch_v<double, 1>(a, smem, s);
      case 2: return launch_v<double, 2>(a, smem, s);
      case 4: return launch_v<double, 4>(a, smem, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace mmk
