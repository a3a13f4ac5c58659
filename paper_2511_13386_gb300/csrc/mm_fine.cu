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
// the per-interface moments as float sums of the lane partials;
// one float flux per interface, added to one cell and subtracted from the
// other, so mass is conserved to float-float rounding.
#include <math.h>
#include <stdio.h>

#include "ff.cuh"
#include "lift.cuh"
#include "mm_internal.h"

namespace mmk {

// Unnormalised float-float forms for the inside of a stencil: the pair
// (s, w) that the sloppy addition of ff.cuh holds before its final Fast2Sum,
// and the product by a float before its Fast2Sum.  |w| may exceed
// ulp(s)/2, and after a cancellation s may carry none of the value, so only
// another unnormalised or sloppy operation or a double-word product may read
// such a pair; the absolute error stays the sloppy addition's, about 2^-47
// of the operands.
__device__ __forceinline__ ff ff_add_raw(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return {s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ ff ff_sub_raw(ff a, ff b) {
  const ff s = two_sum(a.hi, -b.hi);
  return {s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo))};
}
__device__ __forceinline__ ff ff_mul_f_raw(ff a, float b) {
  const float ch = __fmul_rn(a.hi, b);
  const float cl = __fmaf_rn(a.hi, b, -ch);
  return {ch, __fmaf_rn(a.lo, b, cl)};
}

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
  // J from two densities and E
  static __device__ __forceinline__ double flux_J(R r0, R r1, double e, double inv_dx) {
    return (r1 - r0) * inv_dx - e * 0.5 * (r0 + r1);
  }
};

template <>
struct MP<float> {
  using R = ff;
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
  static __device__ __forceinline__ float flux_J(R r0, R r1, float e, float inv_dx) {
    const float dr = ff_sub(r1, r0).hi;
    return dr * inv_dx - e * 0.5f * (r0.hi + r1.hi);
  }
};

// ------------------------------------------------------- column arrays ---

// Per-state column arrays.  They are placed in shared memory in this
// priority order while they fit the kernel's budget; the rest go to a
// per-state block of global memory (one for every state whose column arrays
// do not fit).  The placement is a function of (nx, precision, adaptation,
// budget), computed identically on the host and the device.
enum ColField {
  F_BASE,   // R [kFineThreads]: per-thread prefix bases of the Poisson law;
            //   then int [rows][warps] counts / offsets of the compaction
  F_PAR,    // G [nx][4]: E (value and low part), P = <X>, J per interface:
            //   the sweep constants, and the field of the criteria; while the
            //   criteria run, slot 2 (P of the last step, dead until the new
            //   constants) holds the density derivative (FP32) or a copy of
            //   the density (FP64)
  F_KIN0, F_KIN1, F_KIN2, F_CELL0, F_CELL1,  // uint8 [nx] status flags (adaptation)
  F_RHO,    // R [nx]: density (float-float or double)
  F_FK,     // G [nx]: kinetic interface flux dt/dx <xi g>/eps of the last sweep
  F_MP,     // G [nx]: m+ = <v^+ g> of the last sweep
  F_MM,     // G [nx]: m- = <v^- g> of the last sweep
  F_N2,     // G [nx]: <g^2> per interface (adaptation)
  F_JD,     // 8 B [nx]: centred flux of the criteria (adaptation); with
            //   adaptation the Poisson prefix sums (first half of the macro
            //   phase) and the write list (compaction to the end of the
            //   sweep) share it: the three lifetimes are disjoint
  F_ENDS,   // G [nx][4]: g at the two lowest and the two highest nodes
  F_ELO,    // float [nx]: low part of the float-float field (FP32 path)
  F_S,      // R [nx]: prefix sums of the Poisson law (without adaptation)
  F_COUNT
};

struct ColLayout {
  size_t off[F_COUNT];
  unsigned smem_mask;     // bit f set: field f lives in shared memory
  size_t smem_total;      // bytes in shared memory
  size_t glob_total;      // bytes in global memory per state
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared-memory budget of the column arrays: the fine kernel's dynamic
// shared memory (232,448 B) or the list kernel's (200 KiB), less the
// reduction scratch.
constexpr int kRedSlots = 160;  // reduction scratch entries (8 bytes each)
constexpr size_t kColBudgetFine = 232448 - 8 * kRedSlots;
constexpr size_t kColBudgetList = 200 * 1024 - 8 * kRedSlots;

__host__ __device__ inline ColLayout col_layout(int nx, int gbytes, bool adapt, size_t budget) {
  const size_t n = nx, a = adapt ? 1 : 0;
  size_t sz[F_COUNT];
  const size_t rows = (n + kFineThreads - 1) / kFineThreads;
  sz[F_BASE] = 8 * (size_t)kFineThreads > 4 * rows * (kFineThreads / 32) ? 8 * (size_t)kFineThreads
                                                                          : 4 * rows * (kFineThreads / 32);
  sz[F_PAR] = gbytes * 4 * n;
  sz[F_KIN0] = sz[F_KIN1] = sz[F_KIN2] = sz[F_CELL0] = sz[F_CELL1] = a * n;
  sz[F_RHO] = 8 * n;
  sz[F_FK] = gbytes * n;
  sz[F_MP] = gbytes * n;
  sz[F_MM] = gbytes * n;
  sz[F_N2] = a * gbytes * n;
  sz[F_JD] = a * 8 * n;
  sz[F_ENDS] = gbytes * 4 * n;
  sz[F_ELO] = (gbytes == 4 ? 4 : 0) * n;
  sz[F_S] = (1 - a) * 8 * n;
  ColLayout L;
  L.smem_mask = 0;
  L.smem_total = 0;
  L.glob_total = 0;
  for (int f = 0; f < F_COUNT; ++f) {
    const size_t b = al16(sz[f]);
    if (L.smem_total + b <= budget) {
      L.off[f] = L.smem_total;
      L.smem_total += b;
      L.smem_mask |= 1u << f;
    }
  }
  for (int f = 0; f < F_COUNT; ++f) {
    if (L.smem_mask & (1u << f)) continue;
    L.off[f] = L.glob_total;
    L.glob_total += al16(sz[f]);
  }
  return L;
}

size_t fine_column_bytes(int nx, int nv, int lanes, bool fp32, bool adapt, bool list) {
  (void)nv;
  (void)lanes;
  return col_layout(nx, fp32 ? 4 : 8, adapt, list ? kColBudgetList : kColBudgetFine).glob_total;
}

size_t fine_smem_bytes(int nx, int nv, int lanes, bool fp32, bool adapt, bool list) {
  (void)nv;
  (void)lanes;
  return 8 * (size_t)kRedSlots + col_layout(nx, fp32 ? 4 : 8, adapt, list ? kColBudgetList : kColBudgetFine).smem_total;
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

// Block sum of float-float values (absolute-error additions): warp sums,
// then one warp sums the warp totals and broadcasts the result.
__device__ __forceinline__ ff block_sum_ff(ff v, double* red) {
  for (int m = 16; m > 0; m >>= 1) v = ff_add_abs(v, ff_shfl_xor(v, m));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  ff* r = reinterpret_cast<ff*>(red);
  __syncthreads();
  if (l == 0) r[w] = v;
  __syncthreads();
  if (w == 0) {
    ff t = l < (int)(blockDim.x >> 5) ? r[l] : ff{0.f, 0.f};
    for (int m = 16; m > 0; m >>= 1) t = ff_add_abs(t, ff_shfl_xor(t, m));
    if (l == 0) r[32] = t;
  }
  __syncthreads();
  const ff t = r[32];
  __syncthreads();
  return t;
}

// ------------------------------------------------------------ the kernel --

template <class G>
struct Cols {
  using R = typename MP<G>::R;
  R *rho, *S, *base;
  G *fk, *mp, *mm, *n2, *ends, *par;
  float* elo;
  uint16_t* list;
  double* jd;
  uint8_t *cell0, *cell1, *kin0, *kin1, *kin2;
};

template <class G>
__device__ __forceinline__ Cols<G> carve(unsigned char* sbase, unsigned char* gbase, int nx, bool adapt,
                                         size_t budget) {
  using R = typename MP<G>::R;
  const ColLayout L = col_layout(nx, sizeof(G), adapt, budget);
  auto at = [&](int f) { return ((L.smem_mask >> f) & 1u ? sbase : gbase) + L.off[f]; };
  Cols<G> c;
  c.rho = reinterpret_cast<R*>(at(F_RHO));
  c.S = reinterpret_cast<R*>(at(adapt ? F_JD : F_S));
  c.base = reinterpret_cast<R*>(at(F_BASE));
  c.fk = reinterpret_cast<G*>(at(F_FK));
  c.mp = reinterpret_cast<G*>(at(F_MP));
  c.mm = reinterpret_cast<G*>(at(F_MM));
  c.n2 = reinterpret_cast<G*>(at(F_N2));
  c.ends = reinterpret_cast<G*>(at(F_ENDS));
  c.par = reinterpret_cast<G*>(at(F_PAR));
  c.elo = reinterpret_cast<float*>(at(F_ELO));
  c.list = reinterpret_cast<uint16_t*>(at(F_JD));
  c.jd = reinterpret_cast<double*>(at(F_JD));
  c.cell0 = at(F_CELL0);
  c.cell1 = at(F_CELL1);
  c.kin0 = at(F_KIN0);
  c.kin1 = at(F_KIN1);
  c.kin2 = at(F_KIN2);
  return c;
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Lifting of order L (Def. 1) of one density into g, by the whole block, in
// double: the Poisson law of S^MM (prefix sum, mean-zero gauge), J of S^0,
// then for L = 1 g_{i+1/2,j} = -eps (xi_j M_j - <xi M> M_j) J_{i+1/2}, and
// for L = 2, 3 the higher Chapman-Enskog terms of lift.cuh.  E and J use
// the first 16 nx bytes of `scratch`; orders two and three also use
// scratch2 (16 nx bytes: K, dK) and scratch3 (8 nx bytes: dtJ).
template <class G>
__device__ void lift_block(const FineArgs& A, const double* rho, double rb, G* g, unsigned char* scratch,
                           unsigned char* scratch2, unsigned char* scratch3, double* red) {
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
  if (A.lift_order <= 1) {
    for (unsigned q = tid; q < n; q += T) {
      const unsigned i = q / (unsigned)nv, j = q - i * (unsigned)nv;
      const double Ji = J[i];
      g[q] = (G)(-A.eps * (vM[j] * Ji - A.xiM * Ji * Mj[j]));
    }
    __syncthreads();
    return;
  }
  double* K = reinterpret_cast<double*>(scratch2);
  double* dK = K + nx;
  double* dtJ = reinterpret_cast<double*>(scratch3);
  lift_fields(rho, E, J, K, dK, dtJ, nx, A.inv_dx, red);
  const double* vj = A.vtab + 5 * nv;
  const LiftConsts lc{A.lift_order, A.eps, A.xiM, A.m2, A.mu3};
  for (unsigned q = tid; q < n; q += T) {
    const unsigned i = q / (unsigned)nv, j = q - i * (unsigned)nv;
    g[q] = (G)lift_value(lc, vj[j], Mj[j], E[i], J[i], K[i], dK[i], dtJ[i]);
  }
  __syncthreads();
}

// v[k] = p[k T + threadIdx.x + d] (periodic in nx) for the NR rows of a
// pass over the cells (see fine_state).
template <int NR, int T, class V>
__device__ __forceinline__ void pre_rows(V (&v)[NR], const V* p, int d, int nx) {
#pragma unroll
  for (int k = 0; k < NR; ++k) v[k] = p[wrapi(k * T + (int)threadIdx.x + d, nx)];
}

// F for one state: n_steps steps from (rin, gin); gin == nullptr lifts the
// density first.  buf0/buf1 are the two step buffers (the last step writes
// buf0); the column arrays are carved from colsmem (shared memory, up to
// `budget` bytes) and colglob (global memory, the fields that do not fit).
// Lanes of the sweep's layout for nv velocity nodes (see the host's layout
// rule): two halves of nhp lanes, nhp the power of two >= nv / 2 / VPT.
__host__ __device__ constexpr int pow2_at_least(int x) { return x <= 1 ? 1 : 2 * pow2_at_least((x + 1) / 2); }

// NXC, NVC: the state's nx and nv when fixed at compile time (0: taken from
// the arguments); with them the per-cell loops of the macro phase unroll
// (nx a multiple of the block) and the sweep's layout is constant.
template <class G, int VPT, bool ADAPT, int NXC = 0, int NVC = 0>
__device__ __forceinline__ void fine_state(const FineArgs& A, const double* rin, const G* gin, G* buf0, G* buf1,
                                           double* rout, uint8_t* mout, unsigned char* smem,
                                           unsigned char* colsmem, unsigned char* colglob, size_t budget) {
  using M = MP<G>;
  using R = typename M::R;

  const int tid = threadIdx.x;
  constexpr int NHC = NVC ? NVC / 2 / VPT : 0;
  constexpr int NHPC = NHC ? pow2_at_least(NHC) : 0;
  const int nx = NXC ? NXC : A.nx, nv = NVC ? NVC : A.nv;
  const int nh = NHC ? NHC : A.nh, nhp = NHPC ? NHPC : A.nhp, Lg = NHPC ? 2 * NHPC : A.lanes;
  // every cell c of the state, interleaved over the block (cell c by thread
  // c mod T); unrolled when the number of rows is a constant
  constexpr int NROW = (NXC != 0 && NXC % kFineThreads == 0) ? NXC / kFineThreads : 0;
  int krow = -1;  // row of the cell being visited when the rows unroll (a constant per copy)
  auto cells = [&](auto&& f) {
    if constexpr (NROW != 0) {
#pragma unroll
      for (int k = 0; k < NROW; ++k) {
        krow = k;
        f(k * kFineThreads + (int)threadIdx.x);
      }
    } else {
      for (int c = threadIdx.x; c < nx; c += kFineThreads) f(c);
    }
  };
  // periodic neighbour c + d (|d| <= 3) of a cell visited by cells(): with
  // unrolled rows only the first row can wrap below 0 and only the last one
  // above nx, so the other rows index directly
  auto nb = [&](int c, int d) {
    if constexpr (NROW >= 3) {
      if (d < 0 ? krow > 0 : krow < NROW - 1) return c + d;
    }
    return wrapi(c + d, nx);
  };
  constexpr int T = kFineThreads;
  // Values p[c + d] (periodic) of the cells of every row, read before a pass
  // over the cells when the rows unroll.  The column arrays that did not fit
  // shared memory (the field's low part, the end values) are read through
  // the same kind of pointer as the shared ones, so inside a pass the
  // compiler keeps each row's read behind the previous row's stores: one L2
  // round trip per row.  Read first, the rows' reads are in flight together.
  constexpr int NR = NROW != 0 ? NROW : 1;

  double* red = reinterpret_cast<double*>(smem);
  Cols<G> C = carve<G>(colsmem, colglob, nx, ADAPT, budget);
  if (gin == nullptr) {  // the lifted density goes where the first step does not write
    G* lifted = (A.n_steps & 1) ? buf1 : buf0;
    // E and J of the lifting use the sweep-constant array (16 nx bytes or
    // more), K and dK the end values (16 nx bytes or more), dtJ the prefix
    // sums (8 nx bytes): none written yet
    lift_block<G>(A, rin, A.rho_bar, lifted, reinterpret_cast<unsigned char*>(C.par),
                  reinterpret_cast<unsigned char*>(C.ends), reinterpret_cast<unsigned char*>(C.S), red);
    gin = lifted;
  }

  // ---- ownership of cells in the macro phase: interleaved (cell c by
  // thread c % T, so that a warp touches consecutive cells: conflict-free
  // shared memory, coalesced global memory) everywhere except the first
  // pass of the Poisson prefix sum, where thread t owns the contiguous chunk
  // [t cpt, (t+1) cpt) with cpt a power of two
  int lcpt = 0;
  while ((T << lcpt) < nx) ++lcpt;
  const int cpt = 1 << lcpt;
  const int c0 = min(tid * cpt, nx), c1 = min(c0 + cpt, nx);

  // ---- lane layout of the sweep
  const int lig = tid % Lg;                // lane in group
  const int grp = tid / Lg;
  const int ngrp = T / Lg;
  const bool pos = lig >= nhp;
  const int hl = pos ? lig - nhp : lig;  // lane within its half
  const bool active = hl < nh;
  const int j0 = pos ? nv / 2 + hl * VPT : hl * VPT;
  const bool first_lane = active && j0 == 0;
  const bool last_lane = active && j0 + VPT == nv;
  const int warp_base = (tid & 31) - lig;  // first lane of this group in the warp
  const int src_left = warp_base + ((lig == nhp) ? nh - 1 : max(lig - 1, 0));
  const int src_right = warp_base + ((lig == nh - 1) ? nhp : min(lig + 1, Lg - 1));
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
  // (the FP32 path takes the float copies rounded on the host: a constant
  // the compiler rematerialises under register pressure then costs a
  // parameter load, not a double-to-float conversion on the FP64 pipe)
  constexpr bool F32 = sizeof(G) == 4;
  const G ga = F32 ? (G)A.fa : (G)A.a, gb = F32 ? (G)A.fb : (G)A.b;
  const G g_inv_dx = F32 ? (G)A.f_inv_dx : (G)A.inv_dx, g_inv_dv = F32 ? (G)A.f_inv_dv : (G)A.inv_dv;
  const G g_kflux = F32 ? (G)A.f_kflux : (G)(A.dt_dx * A.inv_eps);  // dt/dx <xi g> / eps
  const G g_fflux = F32 ? (G)A.f_fflux : (G)(-A.dt_dx * A.m2);      // dt/dx (-m2 J)
  R Rdx, Rinv_nx;
  if constexpr (F32) {
    Rdx = ff{A.f_dx, A.f_dx_lo};
    Rinv_nx = ff{A.f_inv_nx, A.f_inv_nx_lo};
  } else {
    Rdx = A.dx;
    Rinv_nx = 1.0 / nx;
  }

  // ---- prologue: density, rho_bar, moments of g_in
  double rb = A.rho_bar;
  {
    double s = 0.0;
    cells([&](int c) {
      const double r = rin[c];
      C.rho[c] = M::c(r);
      s += r;
    });
    if (isnan(rb)) rb = block_sum_d(s, red) / nx;
  }
  const R Rrb = M::c(rb);
  const float rb_f = (float)rb;  // the criteria's float combination

  // Sums of the lane partials of one interface column over each half of the
  // lane group (negative / positive velocities), by shuffles; lane 0 of the
  // group stores the flux, the two half moments and the norm.  Plain sums in
  // the FP32 path too: each lane's partial already carries the rounding of
  // its products of float g, so compensating the sum over the lanes would
  // not make the flux more accurate than its inputs.  Every thread calls it
  // with warp-uniform control flow; `valid` only gates the store.
  auto reduce_store = [&](int i, bool valid, G p, G q) {
#pragma unroll
    for (int m = nhp >> 1; m >= 1; m >>= 1) {
      p += __shfl_xor_sync(0xffffffffu, p, m);
      if constexpr (ADAPT) q += __shfl_xor_sync(0xffffffffu, q, m);
    }
    const int src = warp_base + nhp;
    const G pp = __shfl_sync(0xffffffffu, p, src);
    G qq = G(0);
    if constexpr (ADAPT) qq = __shfl_sync(0xffffffffu, q, src);
    if (valid && lig == 0) {
      // pp: <v^+ g>; p: the sum over the negative velocities
      C.fk[i] = (pp + p) * g_kflux;
      C.mp[i] = pp;
      C.mm[i] = -p;
      if constexpr (ADAPT) C.n2[i] = q + qq;
    }
  };

  for (int base = 0; base < nx; base += ngrp) {  // warp-uniform trip count
    const int i = base + grp;
    const bool valid = i < nx;
    G w1[VPT];
#pragma unroll
    for (int k = 0; k < VPT; ++k) w1[k] = G(0);
    if (active && valid) vload<G, VPT>(w1, gin + (size_t)i * nv + j0);
    G p = 0, q = 0;
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      p += wv[k] * w1[k];
      if constexpr (ADAPT) q += wj[k] * w1[k] * w1[k];
    }
    reduce_store(i, valid, p, q);
    if (valid) {
      if constexpr (VPT >= 2) {
        if (first_lane) { C.ends[4 * i + 0] = w1[0]; C.ends[4 * i + 1] = w1[1]; }
        if (last_lane) { C.ends[4 * i + 2] = w1[VPT - 2]; C.ends[4 * i + 3] = w1[VPT - 1]; }
      } else {
        if (end_slot >= 0) C.ends[4 * i + end_slot] = w1[0];
      }
    }
  }
  if constexpr (ADAPT) {
    cells([&](int c) { C.kin1[c] = 1; C.kin2[c] = 1; });
  }
  __syncthreads();

  uint8_t* cell_cur = C.cell0;   // s^n
  uint8_t* cell_nxt = C.cell1;   // s^{n+1}
  uint8_t* kin_cur = C.kin0;     // interface flags under s^n
  uint8_t* kin_prev = C.kin1;    // under s^{n-1}
  uint8_t* kin_prev2 = C.kin2;   // under s^{n-2}
  int* rint = reinterpret_cast<int*>(red) + 300;  // [0] write count, [1] kinetic count
  int count = nx;                // interfaces to write this step
  long long kin_total = 0;       // kinetic interfaces summed over steps (thread 0)
  const int w = tid >> 5, l = tid & 31;

  // ------------------------------------------------------------ macro A --
  // E, J, criteria/status, write list and sweep constants for step n.
  auto macro_A = [&](bool initial, bool prefix) {
    // the density was last written with interleaved ownership (macro_C or
    // the prologue); the first Poisson pass reads it in contiguous chunks
    __syncthreads();
    if constexpr (ADAPT) {
      if (tid == 0) rint[1] = 0;  // kinetic-interface count of this step
    }
    if (prefix) {  // else E^n was advanced by the Ampere identity in macro_C
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
      C.base[tid] = M::add(rr[64 + w], ex_lane);   // prefix before this thread's chunk
      const R meanS = rr[96];
      __syncthreads();
      cells([&](int c) {  // E^n into slot 0 of the sweep constants (+ low part)
        const R E = M::sub(M::add(C.base[c >> lcpt], C.S[c]), meanS);
        if constexpr (sizeof(G) == 4) {
          C.par[4 * c] = E.hi;
          C.elo[c] = E.lo;
        } else {
          C.par[4 * c] = E;
          C.par[4 * c + 1] = 0.0;
          if constexpr (ADAPT) C.par[4 * c + 2] = C.rho[c];  // density copy for the criteria
        }
      });
      __syncthreads();  // rho final for this step; E of all cells visible
    }

    if constexpr (ADAPT) {
      // criteria of Sec. 2.2 and status update of Sec. 2.3: the remainder R
      // (eq. Remainder with the Table 1 stencils) and the interface norms
      // ||g||_2.  FP64 path in double; FP32 path in float-float (below).
      if constexpr (sizeof(G) == 4) {
        // FP32 path.  GB300 issues FP64 at 1/64 of the FP32 rate, and R is a
        // fourth derivative of the density: its stencils cancel about
        // 1/dx^4 ~ 1e14 of the inputs' size, so plain float is useless and
        // double costs more than the whole g sweep.  The stencil sums run
        // in float-float (~2^-47 absolute error, R accurate to ~1e-5 of the
        // thresholds used); the combination of the cancelled sums into R,
        // and the norms (compared squared), run in float.  Table 1 rows are
        // applied with integer weights: D1 f = (45 e1 - 9 e2 + e3) / 60,
        // D2 f = (270 s1 - 27 s2 + 2 s3 - 490 f0) / 180,
        // D3 f = (-13 e1 + 8 e2 - e3) / 8, with e_k = f_{+k} - f_{-k},
        // s_k = f_{+k} + f_{-k} (then divided by dx^d).  Inside a stencil the
        // pairs stay unnormalised (ff_*_raw); the last operation before a
        // high part is read alone normalises.
        float elo0[NR], elom[NR];  // the field's low part at c and c - 1
        if constexpr (NROW != 0) {
          pre_rows<NR, T>(elo0, C.elo, 0, nx);
          pre_rows<NR, T>(elom, C.elo, -1, nx);
        }
        auto elo_at = [&](int c, int d) {
          if constexpr (NROW != 0) return d == 0 ? elo0[krow] : elom[krow];
          else return C.elo[nb(c, d)];
        };
        ff* Jf = reinterpret_cast<ff*>(C.jd);
        const ff k1 = {A.f_k1, A.f_k1_lo};
        auto rho_f = [&](int c, int d) { return C.rho[nb(c, d)]; };
        ff jsum = {0.f, 0.f};
        cells([&](int c) {
          const ff e1 = ff_sub_raw(rho_f(c, 1), rho_f(c, -1));
          const ff e2 = ff_sub_raw(rho_f(c, 2), rho_f(c, -2));
          const ff e3 = ff_sub_raw(rho_f(c, 3), rho_f(c, -3));
          const ff D1 = ff_mul(ff_add_raw(ff_sub_raw(ff_mul_f_raw(e1, 45.f), ff_mul_f_raw(e2, 9.f)), e3), k1);
          ff Ec = ff_add_raw(ff{C.par[4 * nb(c, -1)], elo_at(c, -1)}, ff{C.par[4 * c], elo_at(c, 0)});
          Ec.hi *= 0.5f;
          Ec.lo *= 0.5f;
          const ff J = ff_sub_abs(D1, ff_mul(Ec, C.rho[c]));
          C.par[4 * c + 2] = D1.hi;  // d rho / dx for the second pass
          Jf[c] = J;
          jsum = ff_add_raw(jsum, J);  // (the block sum normalises)
        });
        const float meanJ = block_sum_ff(jsum, red).hi * A.f_inv_nx;  // (syncs: Jc visible)
        const float rbf = rb_f;
        cells([&](int c) {
          const ff J0 = Jf[c];
          const ff Jm1 = Jf[nb(c, -1)], Jp1 = Jf[nb(c, 1)];
          const ff Jm2 = Jf[nb(c, -2)], Jp2 = Jf[nb(c, 2)];
          const ff Jm3 = Jf[nb(c, -3)], Jp3 = Jf[nb(c, 3)];
          const ff e1 = ff_sub_abs(Jp1, Jm1), e2 = ff_sub_abs(Jp2, Jm2), e3 = ff_sub_abs(Jp3, Jm3);
          // (e_k stay normalised: their high parts form D1 J in float below)
          const ff s1 = ff_add_raw(Jp1, Jm1), s2 = ff_add_raw(Jp2, Jm2), s3 = ff_add_raw(Jp3, Jm3);
          const ff n3 = ff_sub_abs(ff_add_raw(ff_mul_f_raw(e1, -13.f), ff_mul_f_raw(e2, 8.f)), e3);
          const ff n2 = ff_add_abs(ff_add_raw(ff_mul_f_raw(s1, 270.f), ff_mul_f_raw(s2, -27.f)),
                                   ff_add_raw(ff_mul_f_raw(s3, 2.f), ff_mul_f_raw(J0, -490.f)));
          const float d3J = n3.hi * A.f_k3;
          const float d2J = n2.hi * A.f_k2;
          const float d1J = (45.f * e1.hi - 9.f * e2.hi + e3.hi) * A.f_k1;
          const float d1r = C.par[4 * c + 2], jc = J0.hi, rc = C.rho[c].hi;
          const float Ec = 0.5f * (C.par[4 * nb(c, -1)] + C.par[4 * c]);
          const float Rc = -d3J + Ec * d2J + (2.f * rc - 3.f * rbf) * d1J + 2.f * jc * d1r - d1r * (jc - meanJ);
          const bool big_R = A.f_rfac * fabsf(Rc) > A.f_thr_R;
          const bool gl = C.n2[nb(c, -1)] > A.f_thr_g2, gr = C.n2[c] > A.f_thr_g2;
          uint8_t s;
          if (initial) {
            s = (gl || gr || big_R) ? 1 : 0;
            cell_cur[c] = s;
          }
          const uint8_t cur = initial ? s : cell_cur[c];
          if (!cur) s = big_R ? 1 : 0;
          else s = (!gl && !gr && !big_R) ? 0 : 1;
          cell_nxt[c] = s;
        });
      } else {
        const double inv_dx = A.inv_dx;
        auto rho_d = [&](int c) { return C.par[4 * wrapi(c, nx) + 2]; };
        auto E_d = [&](int c) { return C.par[4 * wrapi(c, nx)]; };
        double jsum = 0.0;
        cells([&](int c) {
          double d1 = 0.0;
          for (int k = -3; k <= 3; ++k) d1 += kFD[0][k + 3] * rho_d(c + k);
          d1 *= inv_dx;
          const double Ec = 0.5 * (E_d(c - 1) + E_d(c));
          C.jd[c] = d1 - Ec * rho_d(c);
          jsum += C.jd[c];
        });
        const double meanJ = block_sum_d(jsum, red) / nx;  // (syncs: Jc visible)
        const double r2 = 1.0 / (A.dx * A.dx), r3 = r2 / A.dx;
        cells([&](int c) {
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
          const double nl = sqrt((double)C.n2[wrapi(c - 1, nx)]), nr = sqrt((double)C.n2[c]);
          uint8_t s;
          if (initial) {
            s = (nl > A.thr_g || nr > A.thr_g || big_R) ? 1 : 0;
            cell_cur[c] = s;
          }
          const uint8_t cur = initial ? s : cell_cur[c];
          if (!cur) s = big_R ? 1 : 0;
          else s = (nl <= A.thr_g && nr <= A.thr_g && !big_R) ? 0 : 1;
          cell_nxt[c] = s;
        });
      }
      __syncthreads();  // cell_cur of all cells visible

      // interface flags under s^n; an interface is written while it is
      // kinetic and for the two steps after it turns fluid, so that both
      // step buffers hold its zeros.  Compaction of the interfaces to write,
      // in increasing order: rows of T cells (cell k T + tid), one ballot
      // per warp and row, an exclusive scan of the per-(row, warp) counts,
      // then each flagged cell's slot from the popcount of the lanes below
      // it.
      constexpr int NW = T / 32;
      const int nrow = (nx + T - 1) / T;
      int* cnt = reinterpret_cast<int*>(C.base);  // [nrow][NW]
      int nk = 0;
      for (int k = 0; k < nrow; ++k) {
        const int c = k * T + tid;
        bool wr = false;
        if (c < nx) {
          const uint8_t kf = cell_cur[c] | cell_cur[wrapi(c + 1, nx)];
          kin_cur[c] = kf;
          nk += kf;
          wr = (kf | kin_prev[c] | kin_prev2[c]) != 0;
        }
        const unsigned b = __ballot_sync(0xffffffffu, wr);
        if (l == 0) cnt[k * NW + w] = __popc(b);
      }
      nk = __reduce_add_sync(0xffffffffu, nk);
      if (l == 0) atomicAdd(&rint[1], nk);
      __syncthreads();
      if (w == 0) {
        const int ne = nrow * NW, per = (ne + 31) / 32;
        const int q0 = min(l * per, ne), q1 = min(q0 + per, ne);
        int sum = 0;
        for (int q = q0; q < q1; ++q) sum += cnt[q];
        int inc = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, inc, d);
          if (l >= d) inc += t;
        }
        int run = inc - sum;
        for (int q = q0; q < q1; ++q) {
          const int v = cnt[q];
          cnt[q] = run;
          run += v;
        }
        if (l == 31) rint[0] = inc;
      }
      __syncthreads();
      count = rint[0];
      for (int k = 0; k < nrow; ++k) {
        const int c = k * T + tid;
        const bool wr = c < nx && (kin_cur[c] | kin_prev[c] | kin_prev2[c]);
        const unsigned b = __ballot_sync(0xffffffffu, wr);
        if (wr) C.list[cnt[k * NW + w] + __popc(b & ((1u << l) - 1u))] = (uint16_t)c;
      }
    } else {
      count = nx;
      if (tid == 0) kin_total += nx;
    }

    // J and the sweep constants: E+/dv, E-/dv, P = <X>, J
    float4 ends4[NR];  // FP32, rows unrolled: the end values and the
    float eloc[NR];    // field's low part of every row, read first
    if constexpr (F32 && NROW != 0) {
      pre_rows<NR, T>(ends4, reinterpret_cast<const float4*>(C.ends), 0, nx);
      pre_rows<NR, T>(eloc, C.elo, 0, nx);
    }
    cells([&](int c) {
      const int cl = nb(c, -1), cr = nb(c, 1);
      G* pr = C.par + 4 * c;
      const G e = pr[0];
      const G ep = e > G(0) ? e : G(0), em = e < G(0) ? -e : G(0);
      const G pm = ((C.mp[c] - C.mp[cl]) - (C.mm[cr] - C.mm[c])) * g_inv_dx;
      G en[4];
      if constexpr (sizeof(G) == 4) {
        float4 e4;
        if constexpr (NROW != 0) e4 = ends4[krow];
        else e4 = *reinterpret_cast<const float4*>(C.ends + 4 * c);
        en[0] = e4.x; en[1] = e4.y; en[2] = e4.z; en[3] = e4.w;
      } else {
        for (int q = 0; q < 4; ++q) en[q] = C.ends[4 * c + q];
      }
      const G gend = (G)0.5 * ((ep * en[2] - em * en[3]) - (ep * en[0] - em * en[1]));
      pr[2] = pm + gend;
      if constexpr (sizeof(G) == 4) {
        // J in float-float: the fluid flux -m2 J feeds the density, and a
        // float-rounded flux would leave cell-to-cell noise of ~1e-7 |F| in
        // it, which the fourth derivative inside the remainder R amplifies
        // by ~nx^4 (past the thresholds at nx >= 2048).  The sweep reads the
        // high part (slot 3); the low part replaces the field's (slot 1,
        // dead after the criteria).
        const ff r0 = C.rho[c], r1 = C.rho[cr];
        ff avg = ff_add_raw(r0, r1);  // (read only by the product below)
        avg.hi *= 0.5f;
        avg.lo *= 0.5f;
        float el;
        if constexpr (NROW != 0) el = eloc[krow];
        else el = C.elo[c];
        const ff J = ff_sub_abs(ff_mul_f_raw(ff_sub_raw(r1, r0), g_inv_dx), ff_mul(ff{pr[0], el}, avg));
        pr[3] = J.hi;
        pr[1] = J.lo;
      } else {
        pr[3] = M::flux_J(C.rho[c], C.rho[cr], e, g_inv_dx);
      }
    });
    __syncthreads();
    if constexpr (ADAPT) {
      if (tid == 0) kin_total += rint[1];
    }
  };

  // ------------------------------------------------------------ macro C --
  // density update from the fluxes of the new g: one flux per interface
  // (kinetic: dt/dx <xi g>/eps, fluid: dt/dx (-m2 J)), or the cell-based
  // rule of S^HMM when flux_rule == 1.
  // fluxes in the density's precision (float-float in the FP32 path): the
  // kinetic flux of the last sweep, or the fluid flux dt/dx (-m2 J) from J
  // (slot 3, and its low part in slot 1 in the FP32 path)
  auto flux_kin = [&](int c) -> R {
    if constexpr (sizeof(G) == 4) return ff{C.fk[c], 0.f};
    else return C.fk[c];
  };
  auto flux_fluid = [&](int c) -> R {
    if constexpr (sizeof(G) == 4) return ff_mul_f(ff{C.par[4 * c + 3], C.par[4 * c + 1]}, g_fflux);
    else return g_fflux * C.par[4 * c + 3];
  };
  auto is_kin = [&](int c) { return ADAPT ? kin_cur[c] != 0 : true; };
  // FP32 path with one flux per interface: the field is advanced with the
  // density instead of re-solving the Poisson law at the next step.  Summing
  // the density update over the cells m <= c telescopes the fluxes, so the
  // law of S^MM at n+1 is exactly E^{n+1}_c = E^n_c - dx (F_c - mean F).
  // Pass 1 forms every interface flux in float-float (high part over the
  // kinetic flux, low part over the low part of J, both read only here);
  // pass 2 updates the density and the field.
  const bool ampere = F32 && A.flux_rule == 0;
  auto macro_C_ampere = [&]() {
    if constexpr (F32) {
      ff fsum = {0.f, 0.f};
      cells([&](int c) {
        const ff F = is_kin(c) ? flux_kin(c) : flux_fluid(c);
        C.fk[c] = F.hi;
        C.par[4 * c + 1] = F.lo;
        fsum = ff_add_raw(fsum, F);  // (the block sum normalises)
      });
      const ff Fbar = ff_mul(block_sum_ff(fsum, red), Rinv_nx);  // (syncs: fluxes visible)
      const ff mdx = {-Rdx.hi, -Rdx.lo};
      float eloc[NR];  // rows unrolled: the field's low part of every row, read first
      if constexpr (NROW != 0) pre_rows<NR, T>(eloc, C.elo, 0, nx);
      // sums of terms that are small against the density and the field:
      // the absolute-error form (error ~2^-47 of the operands) suffices
      cells([&](int c) {
        const int cl = nb(c, -1);
        const ff Fl = {C.fk[cl], C.par[4 * cl + 1]}, Fc = {C.fk[c], C.par[4 * c + 1]};
        C.rho[c] = ff_add_abs(C.rho[c], ff_sub_raw(Fl, Fc));
        float el;
        if constexpr (NROW != 0) el = eloc[krow];
        else el = C.elo[c];
        const ff E = ff_add_abs(ff{C.par[4 * c], el}, ff_mul(ff_sub_raw(Fc, Fbar), mdx));
        C.par[4 * c] = E.hi;
        C.elo[c] = E.lo;
      });
    }
  };
  auto macro_C = [&]() {
    if (ampere) {
      macro_C_ampere();
    } else if (A.flux_rule == 0) {
      // each interface flux is evaluated by both of its cells, from the same
      // inputs, so the two evaluations are bitwise equal and mass telescopes
      cells([&](int c) {
        const int cl = wrapi(c - 1, nx);
        const R Fl = is_kin(cl) ? flux_kin(cl) : flux_fluid(cl);
        const R Fc = is_kin(c) ? flux_kin(c) : flux_fluid(c);
        C.rho[c] = M::sub(M::add(C.rho[c], Fl), Fc);
      });
    } else {
      cells([&](int c) {
        const int cl = wrapi(c - 1, nx);
        R Fr, Fl;
        if (!ADAPT || cell_cur[c]) {
          Fr = is_kin(c) ? flux_kin(c) : M::zero();
          Fl = is_kin(cl) ? flux_kin(cl) : M::zero();
        } else {
          Fr = flux_fluid(c);
          Fl = flux_fluid(cl);
        }
        C.rho[c] = M::sub(M::add(C.rho[c], Fl), Fr);
      });
    }
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
    // (in flight); afterwards P receives g(i+3).  (A five-column ring with
    // two columns in flight measured no faster at the hybrid workload.)
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
      G psum = 0, nsum = 0;
      if (valid) {
        const bool kin = ADAPT ? (kin_cur[i] != 0) : true;
        G out[VPT];
        if (kin) {
          const float4* pr4 = reinterpret_cast<const float4*>(C.par + 4 * i);
          G Ep, Em, Pp, Jv;
          G Ev;
          if constexpr (sizeof(G) == 4) {
            const float4 q = *pr4;
            Ev = q.x; Pp = q.z; Jv = q.w;
          } else {
            const G* pr = C.par + 4 * i;
            Ev = pr[0]; Pp = pr[2]; Jv = pr[3];
          }
          Ep = Ev > G(0) ? Ev * g_inv_dv : G(0);
          Em = Ev < G(0) ? -Ev * g_inv_dv : G(0);
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
        if constexpr (VPT >= 2) {
          if (first_lane) { C.ends[4 * i + 0] = out[0]; C.ends[4 * i + 1] = out[1]; }
          if (last_lane) { C.ends[4 * i + 2] = out[VPT - 2]; C.ends[4 * i + 3] = out[VPT - 1]; }
        } else {
          if (end_slot >= 0) C.ends[4 * i + end_slot] = out[0];
        }
      }
      reduce_store(i, valid, psum, nsum);
    };
    for (int e = e0; e < e0 + epg; e += 4) {
      body(e + 0, R0, R1, R2, R3);
      body(e + 1, R1, R2, R3, R0);
      body(e + 2, R2, R3, R0, R1);
      body(e + 3, R3, R0, R1, R2);
    }
  };

  // ------------------------------------------------------------ step loop --
  macro_A(true, true);
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
    if (s + 1 < A.n_steps) macro_A(false, !ampere);
    src = dst;
  }
  __syncthreads();

  // ---- epilogue
  int bad = 0;
  cells([&](int c) {
    const double r = M::tod(C.rho[c]);
    rout[c] = r;
    if (!isfinite(r)) bad = 1;
    if (mout) mout[c] = ADAPT ? cell_cur[c] : 1;
  });
  if (bad) atomicExch(A.status, (int)MM_ERR_UNSTABLE);
  if (tid == 0 && A.kin_count) atomicAdd(A.kin_count, (unsigned long long)kin_total * (unsigned long long)nv);
}

// One CTA per state of a uniform batch (NXC, NVC: see fine_state).
template <class G, int VPT, bool ADAPT, int NXC = 0, int NVC = 0>
__global__ void __launch_bounds__(kFineThreads, 1) fine_kernel(const FineArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t st = blockIdx.x;
  const size_t sz = (size_t)A.nx * A.nv;
  unsigned char* colglob =
      A.col_ws ? reinterpret_cast<unsigned char*>(A.col_ws) + st * A.col_ws_stride : nullptr;
  fine_state<G, VPT, ADAPT, NXC, NVC>(A, A.rho_in + st * A.nx, reinterpret_cast<const G*>(A.g_in) + st * sz,
                            reinterpret_cast<G*>(A.g_buf0) + st * sz, reinterpret_cast<G*>(A.g_buf1) + st * sz,
                            A.rho_out + st * A.nx, A.mask_out ? A.mask_out + st * A.nx : nullptr, smem,
                            smem + 8 * kRedSlots, colglob, kColBudgetFine);
}

// Persistent work-list kernel: each CTA takes (solve, slice) items from a
// global counter until the list is exhausted (dynamic scheduling of uneven
// fine propagations; the list is sorted by decreasing cost on the host).
// An item propagates rho^{n,k} of its solve (g from slice 0's data, or
// lifted from the density) and writes F(rho)^{n+1}.  The step buffers and
// the column arrays that do not fit shared memory are per-CTA workspace
// reused from item to item.
template <class G, int VPT, bool ADAPT>
__global__ void __launch_bounds__(kFineThreads, 1)
    fine_list_kernel(const FineListSolve* solves, const FineListItem* items, int n_items, int* next,
                     unsigned char* ws, size_t ws_g, size_t ws_col) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ __align__(16) FineArgs s_args;
  unsigned char* mine = ws + (size_t)blockIdx.x * (2 * ws_g + ws_col);
  G* b0 = reinterpret_cast<G*>(mine);
  G* b1 = reinterpret_cast<G*>(mine + ws_g);
  unsigned char* colglob = ws_col ? mine + 2 * ws_g : nullptr;
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
    fine_state<G, VPT, ADAPT>(s_args, S->rho + (size_t)it.slice * nx, gin, b0, b1,
                              S->frho + (size_t)(it.slice + 1) * nx, nullptr, smem, smem + 8 * kRedSlots,
                              colglob, kColBudgetList);
    __syncthreads();  // before the next item overwrites s_args, s_item and the buffers
  }
}

// ---------------------------------------------------------------- launch --

// dry: configure (and so load) the instance without launching it.
template <class G, int VPT, bool ADAPT, int NXC = 0, int NVC = 0>
static cudaError_t launch_t(const FineArgs& a, size_t smem, cudaStream_t s, bool dry) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(fine_kernel<G, VPT, ADAPT, NXC, NVC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (dry) return cudaSuccess;
  fine_kernel<G, VPT, ADAPT, NXC, NVC><<<a.batch, kFineThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Instances with the shape fixed at compile time: FP32 g, 8 nodes per lane,
// Nx = 4096 and Nv = 128 (the hybrid-adaptation grid); every other shape
// takes the runtime-shape kernel.
template <class G, int VPT>
static cudaError_t launch_v(const FineArgs& a, size_t smem, cudaStream_t s, bool dry) {
  if constexpr (sizeof(G) == 4 && VPT == 8) {
    if (a.nx == 4096 && a.nv == 128)
      return a.adapt ? launch_t<G, VPT, true, 4096, 128>(a, smem, s, dry)
                     : launch_t<G, VPT, false, 4096, 128>(a, smem, s, dry);
  }
  return a.adapt ? launch_t<G, VPT, true>(a, smem, s, dry) : launch_t<G, VPT, false>(a, smem, s, dry);
}

template <class G, int VPT, bool ADAPT>
static cudaError_t launch_list_t(const FineList& L, size_t smem, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(fine_list_kernel<G, VPT, ADAPT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  fine_list_kernel<G, VPT, ADAPT><<<L.grid, kFineThreads, smem, s>>>(L.solves, L.items, L.n_items, L.next,
                                                                     L.ws, L.ws_g, L.ws_col);
  return cudaGetLastError();
}

cudaError_t launch_fine_list(const FineList& L, bool fp32, bool adapt, size_t smem, cudaStream_t s) {
  if (fp32) return adapt ? launch_list_t<float, 8, true>(L, smem, s) : launch_list_t<float, 8, false>(L, smem, s);
  return adapt ? launch_list_t<double, 4, true>(L, smem, s) : launch_list_t<double, 4, false>(L, smem, s);
}

static cudaError_t fine_dispatch(const FineArgs& args, int vpt, bool fp32, size_t smem, cudaStream_t s,
                                 bool dry) {
  FineArgs a = args;
  fine_args_floats(a);
  if (fp32) {
    switch (vpt) {
      case 1: return launch_v<float, 1>(a, smem, s, dry);
      case 2: return launch_v<float, 2>(a, smem, s, dry);
      case 4: return launch_v<float, 4>(a, smem, s, dry);
      case 8: return launch_v<float, 8>(a, smem, s, dry);
    }
  } else {
    switch (vpt) {
      case 1: return launch_v<double, 1>(a, smem, s, dry);
      case 2: return launch_v<double, 2>(a, smem, s, dry);
      case 4: return launch_v<double, 4>(a, smem, s, dry);
      case 8: return launch_v<double, 8>(a, smem, s, dry);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fine(const FineArgs& args, int vpt, bool fp32, size_t smem, cudaStream_t s) {
  return fine_dispatch(args, vpt, fp32, smem, s, false);
}

cudaError_t fine_stream_preload(const FineArgs& a, int vpt, bool fp32) {
  return fine_dispatch(a, vpt, fp32, 0, nullptr, true);
}

}  // namespace mmk
