// Fine propagator F = S^MM (Sec. 2.3) with the slice states resident in
// shared memory: FP32 g, every cell kinetic, one flux per interface.
//
// A state (rho[nx], g[nx][nv]) is split over a thread-block cluster of C
// CTAs (C = 1, 2, 4 or 8, the smallest that fits the state into the
// cluster's shared memory); CTA r owns the cells and interfaces
// [r nx/C, (r+1) nx/C).  g never leaves shared memory between the first
// and the last step of the launch, so HBM and L2 see only the initial load
// and the final store; each step is bound by shared-memory and FP32 issue.
//
// Per step n -> n+1:
//   sweep      every group of `LG` lanes updates a run of interface columns
//              in place (upwind v d_x g, E d_v g, (I - Pi), relaxation),
//              from a register ring holding the old columns i-1, i, i+1 and
//              a prefetch; the old columns it needs from the neighbouring
//              groups come from stashes that each group fills right after
//              its sweep of the step before; the per-lane partial moments
//              <w v g> of the new column are stored;
//   macro (i)  per cell: the interface flux F = (dt/dx) <xi g>/eps as the
//              sum of the partials, m+- = <v^+- g>, the warp
//              sums of F, and the boundary values the neighbouring warps and
//              CTAs need; the CTA's first and last new columns are copied
//              into the neighbouring CTAs' halo buffers;
//   exchange   one barrier per step (cluster-wide when C > 1); every
//              exchange buffer is double-buffered by step parity, so one
//              barrier separates each write from its read and the next write
//              (with runs as long as the lane groups are wide, where every
//              thread's cell is swept by its own warp, that is the step's
//              only block-wide barrier);
//   macro (ii) per cell: rho^{n+1} = rho^n + F_{i-1/2} - F_{i+1/2}; the
//              field by the discrete Ampere identity (below); J, P = <X> and
//              the sweep constants of the next step.
//
// The Poisson law of S^MM, E_{i+1/2} - E_{i-1/2} = (rho_i - rho_bar) dx with
// a mean-zero gauge, is solved once at entry (prefix sum in double).  After
// that, summing the density update over cells m <= i telescopes the fluxes,
// so the same law at n+1 is exactly
//   E^{n+1}_{i+1/2} = E^n_{i+1/2} - dx (F_{i+1/2} - mean_k F_{k+1/2}),
// which needs one global sum per step instead of a prefix sum (it relies on
// the one-flux-per-interface density update, so the cell-based rule keeps
// the streaming kernel).
//
// Precision: g, the sweep and the per-lane partials in float; the density
// and the field in float-float; the flux as a float sum of the partials.
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "ff.cuh"
#include "mm_internal.h"

namespace cg = cooperative_groups;

namespace mmk {

namespace {

constexpr int T = kResThreads;
constexpr int NW = T / 32;
constexpr int VPT = 8;  // velocity nodes per lane (two 16-byte chunks)

// Shared-memory map (byte offsets).  g columns are stored with the lane's
// two 16-byte chunks interleaved across the group (chunk q of lane l at
// (q * LG + l) * 16), so that eight consecutive lanes touch 128 contiguous
// bytes per access and no bank is hit twice.  The per-column partial moments
// (one row per lane) and the four end values g_0, g_1, g_{nv-2}, g_{nv-1}
// (four more rows) are stored transposed with a row stride of n + 1 floats:
// a group writes one column of it, a thread of the macro phase reads one
// row entry per value, both without bank conflicts.  The per-interface sweep
// constants are stored with one 16-byte pad after each run of R columns, so
// that the groups of a warp, which read the same position of their runs at
// once, hit different banks.
struct ResMap {
  unsigned g, halo, stash, stashl, part, par, wfirst, wlast, xch, pro, red, total;
  unsigned xch_stride;  // bytes per parity in xch
};

__host__ __device__ inline unsigned up16(unsigned x) { return (x + 15u) & ~15u; }

__host__ __device__ inline ResMap res_map(int n, int nv, int lanes, int C) {
  ResMap m;
  unsigned o = 0;
  m.g = o;      o = up16(o + 4u * n * nv);
  m.halo = o;   o = up16(o + 4u * 4 * nv);          // [parity][left, right][nv]
  m.part = o;   o = up16(o + 4u * (lanes + 4) * (n + 1));  // [lanes + 4][n + 1], see below
  m.stash = o;  o = up16(o + 4u * 2 * (T / lanes) * nv);  // [parity][group]: next group's old first column
  m.stashl = o; o = up16(o + 4u * 2 * NW * nv);       // [parity][warp]: previous warp's old last column
  m.par = o;    o = up16(o + 16u * (n + n / ((unsigned)n / (T / lanes))));  // padded, see below
  m.wfirst = o; o = up16(o + 2 * 16u * NW);         // [parity][warp]: F, m-, rho.hi, rho.lo
  m.wlast = o;  o = up16(o + 2 * 16u * NW);         // [parity][warp]: F, m+
  m.xch_stride = up16(16u + 4u * C * NW);           // xL(F, m+), xR(F, m-), sums
  m.xch = o;    o = up16(o + 2u * m.xch_stride);
  m.pro = o;    o = up16(o + 32u * C);              // entry exchange, per rank
  m.red = o;    o = up16(o + 16u * NW);
  m.total = o;
  return m;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// Remote (DSMEM) view of this CTA's shared address `p` in cluster rank r.
template <class P>
__device__ __forceinline__ P* remote(P* p, int r) {
  return cg::this_cluster().map_shared_rank(p, r);
}

__device__ __forceinline__ void cluster_or_block_sync(int C) {
  if (C > 1) cg::this_cluster().sync();
  else __syncthreads();
}

// Block-wide inclusive scan (double) of one value per thread; returns the
// inclusive prefix and writes the block total to *tot.  red: NW doubles.
__device__ double block_scan_d(double v, double* red, double* tot) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int d = 1; d < 32; d <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, d);
    if (l >= d) v += t;
  }
  __syncthreads();
  if (l == 31) red[w] = v;
  __syncthreads();
  double off = 0.0, all = 0.0;
  for (int q = 0; q < NW; ++q) {
    if (q < w) off += red[q];
    all += red[q];
  }
  __syncthreads();
  *tot = all;
  return off + v;
}

// RC: the run length R of a lane group when it is known at compile time
// (the sweep loop then unrolls completely, without runtime branches), 0
// when it is taken from the shape at run time; CC likewise for the cluster
// size (the loops over the cluster's CTAs unroll).
template <int LG, int RC, int CC>
__global__ void __launch_bounds__(T, 2) fine_resident_kernel(const FineArgs A, int C_arg) {
  const int C = CC ? CC : C_arg;
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int HALF = LG / 2;
  constexpr int NGRP = T / LG;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // shape: nv = 8 LG always; with the run length fixed, the CTA's cells
  // n = R x (groups) too, and with the cluster size also nx = n C
  const int nv = LG * VPT;
  const int n = RC ? RC * NGRP : A.nx / C;  // cells (and interfaces) of this CTA
  const int nx = (RC && CC) ? n * CC : A.nx;
  const int r = C > 1 ? (int)cg::this_cluster().block_rank() : 0;
  // work item of this cluster: a chunk of A.n_steps steps of one state
  // (items are numbered chunk-major, item = chunk x batch + state, so a
  // launch never holds two chunks of a state and its states wrap around the
  // batch at most once); the first chunk of a state reads the input
  const int item = A.res_item0 + (int)(blockIdx.x / C);
  const bool from_input = A.res_from_input && item < A.batch;
  const int stx = A.res_state0 + (int)(blockIdx.x / C);  // state, before the wrap
  const int a = r * n;                   // first global cell of this CTA
  const int rl = (r + C - 1) % C, rr = (r + 1) % C;
  const int nwc = n >> 5;                // warps that own cells
  const bool has_cell = tid < n;
  const int R = RC ? RC : n / NGRP;      // columns per group
  const bool warp_local = R == LG;       // thread t's cell t lies in its own group's run

  const ResMap Mp = res_map(n, nv, LG, C);
  float* g = reinterpret_cast<float*>(smem + Mp.g);
  float* halo = reinterpret_cast<float*>(smem + Mp.halo);
  float* part = reinterpret_cast<float*>(smem + Mp.part);
  float* stash = reinterpret_cast<float*>(smem + Mp.stash);
  float* stashl = reinterpret_cast<float*>(smem + Mp.stashl);
  float* par = reinterpret_cast<float*>(smem + Mp.par);
  float* wfirst = reinterpret_cast<float*>(smem + Mp.wfirst);
  float* wlast = reinterpret_cast<float*>(smem + Mp.wlast);
  double* pro = reinterpret_cast<double*>(smem + Mp.pro);
  double* red = reinterpret_cast<double*>(smem + Mp.red);
  auto xch = [&](int p) { return reinterpret_cast<float*>(smem + Mp.xch + p * Mp.xch_stride); };

  // ---- sweep lane layout: lane l of a group owns v nodes [8 l, 8 l + 8)
  const int lig = tid & (LG - 1);
  const int grp = tid / LG;
  const bool pos = lig >= HALF;
  const bool first_lane = lig == 0, last_lane = lig == LG - 1;
  const int wbase = (tid & 31) - lig;
  const int src_left = wbase + (lig > 0 ? lig - 1 : 0);
  const int src_right = wbase + (lig < LG - 1 ? lig + 1 : LG - 1);
  const int i0 = grp * R;
  const unsigned ch0 = 4u * lig, ch1 = 4u * (LG + lig);   // chunk offsets in a column (floats)

  // per-node constants: alpha = a - b|v|/dx, beta = b|v|/dx, M, v M, w v
  float al[VPT], be[VPT], Mj[VPT], xM[VPT], wv[VPT];
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    const int j = VPT * lig + k;
    be[k] = A.fb * A.vtab_f[0 * nv + j];
    al[k] = A.fa - be[k];
    Mj[k] = A.vtab_f[1 * nv + j];
    xM[k] = A.vtab_f[2 * nv + j];
    wv[k] = A.vtab_f[3 * nv + j];
  }
  const float f_b = A.fb, f_inv_dx = A.f_inv_dx, f_inv_dv = A.f_inv_dv;
  const float f_kflux = A.f_kflux, f_dx = A.f_dx, f_inv_nx = A.f_inv_nx;

  auto col = [&](int i) { return g + (unsigned)i * (unsigned)nv; };
  auto ldcol = [&](float (&v)[VPT], const float* c) {
    const float4 p = ld4(c + ch0), q = ld4(c + ch1);
    v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w;
    v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
  };
  auto stcol = [&](float* c, const float (&v)[VPT]) {
    st4(c + ch0, make_float4(v[0], v[1], v[2], v[3]));
    st4(c + ch1, make_float4(v[4], v[5], v[6], v[7]));
  };
  // partial moment <w v g> of one lane
  auto lane_partial = [&](const float (&v)[VPT]) {
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int k = 0; k < VPT; k += 2) {
      p0 = __fmaf_rn(wv[k], v[k], p0);
      p1 = __fmaf_rn(wv[k + 1], v[k + 1], p1);
    }
    return p0 + p1;
  };
  const unsigned PS = n + 1;  // row stride of part
  auto put_partial = [&](int i, float p, const float (&v)[VPT]) {
    part[lig * PS + i] = p;
    if (first_lane) {
      part[(LG + 0) * PS + i] = v[0];
      part[(LG + 1) * PS + i] = v[1];
    }
    if (last_lane) {
      part[(LG + 2) * PS + i] = v[VPT - 2];
      part[(LG + 3) * PS + i] = v[VPT - 1];
    }
  };

  // ------------------------------------------------------------ entry ---
  const size_t sbase = (size_t)(stx >= A.batch ? stx - A.batch : stx) * nx;
  // chunk 0 starts from the input; later chunks from the previous chunk's
  // output, which they overwrite in place (the whole state is in shared
  // memory before the first write)
  const float* gin = reinterpret_cast<const float*>(from_input ? A.g_in : A.g_buf0) + sbase * nv;
  // own columns, and (cluster) the two neighbour columns of step 0
  for (int i = grp; i < n; i += NGRP) {
    const float* s = gin + (size_t)(a + i) * nv + VPT * lig;
    const float4 p = *reinterpret_cast<const float4*>(s), q = *reinterpret_cast<const float4*>(s + 4);
    st4(col(i) + ch0, p);
    st4(col(i) + ch1, q);
  }
  if (C > 1 && grp < 2) {
    const int gi = grp == 0 ? (a + nx - 1) % nx : (a + n) % nx;
    const float* s = gin + (size_t)gi * nv + VPT * lig;
    float* d = halo + (unsigned)(grp) * nv;  // parity 0: [left, right]
    st4(d + ch0, *reinterpret_cast<const float4*>(s));
    st4(d + ch1, *reinterpret_cast<const float4*>(s + 4));
  }

  // density, rho_bar and the entry field (prefix sum in double)
  const double* rin = (from_input ? A.rho_in : A.rho_out) + sbase;
  const double rc = has_cell ? rin[a + tid] : 0.0;
  double rb = A.rho_bar;
  if (isnan(rb)) {
    double tot;
    block_scan_d(rc, red, &tot);
    if (tid == 0)
      for (int q = 0; q < C; ++q) (C > 1 ? remote(pro, q) : pro)[4 * r] = tot;
    cluster_or_block_sync(C);
    double s = 0.0;
    for (int q = 0; q < C; ++q) s += pro[4 * q];
    rb = s / nx;
    cluster_or_block_sync(C);  // pro is reused below
  }
  ff rho = ff_from_double(rc), E;
  {
    const double d = has_cell ? (rc - rb) * A.dx : 0.0;
    double t1, t2;
    const double S = block_scan_d(d, red, &t1);
    block_scan_d(has_cell ? (double)(nx - (a + tid)) * d : 0.0, red, &t2);
    if (tid == 0)
      for (int q = 0; q < C; ++q) {
        double* dst = C > 1 ? remote(pro, q) : pro;
        dst[4 * r + 1] = t1;
        dst[4 * r + 2] = t2;
      }
    cluster_or_block_sync(C);
    double base = 0.0, mean = 0.0;
    for (int q = 0; q < C; ++q) {
      if (q < r) base += pro[4 * q + 1];
      mean += pro[4 * q + 2];
    }
    E = ff_from_double(base + S - mean / nx);
  }
  // ghost density of the first cell of the right neighbour (cluster)
  ff ghost = ff_from_double(C > 1 && tid == n - 1 ? rin[(a + n) % nx] : 0.0);

  // partials of g^0
  for (int i = grp; i < n; i += NGRP) {
    float v[VPT];
    ldcol(v, col(i));
    put_partial(i, lane_partial(v), v);
  }
  __syncthreads();

  // ------------------------------------------------------ macro phases ---
  float Fc = 0.f, mp = 0.f, mm = 0.f;   // flux, m+, m- of this thread's interface

  // (i): from the partials of the new g; F = 0 at entry (no update)
  auto macro_i = [&](int p, bool with_flux) {
    if (w < nwc) {
      const float* pp = part + tid;
      // m-: negative-velocity lanes, m+: positive ones; the flux is their
      // sum.  Plain float sums: each lane's partial already carries the
      // rounding of its eight products of float g, so a compensated sum over
      // the lanes would not make the flux more accurate than its inputs
      float sp = 0.f, sm = 0.f;
      float t[LG];
#pragma unroll
      for (int q = 0; q < LG; ++q) t[q] = pp[q * PS];
#pragma unroll
      for (int q = 0; q < LG; ++q) {
        if (q >= HALF) sp += t[q];
        else sm += t[q];
      }
      mp = sp;
      mm = -sm;
      Fc = with_flux ? __fmul_rn(__fadd_rn(sp, sm), f_kflux) : 0.f;
      float ws = Fc;
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, m);
      float* X = xch(p);
      if (lane == 0) {
        st4(wfirst + 4 * (p * NW + w), make_float4(Fc, mm, rho.hi, rho.lo));
        if (C > 1)
          for (int q = 0; q < C; ++q) remote(X, q)[4 + r * NW + w] = ws;
        else
          X[4 + w] = ws;
      }
      if (lane == 31) *reinterpret_cast<float2*>(wlast + 4 * (p * NW + w)) = make_float2(Fc, mp);
      if (C > 1 && tid == 0) *reinterpret_cast<float2*>(remote(X, rl) + 2) = make_float2(Fc, mm);
      if (C > 1 && tid == n - 1) *reinterpret_cast<float2*>(remote(X, rr)) = make_float2(Fc, mp);
    }
    // the CTA's first (last) column becomes the right (left) neighbour
    // column of the left (right) CTA for the next step
    if (C > 1 && with_flux) {
      if (warp_local) {  // by the groups that wrote them
        if (grp == 0 || grp == NGRP - 1) {
          const bool first = grp == 0;
          const float* c = col(first ? 0 : n - 1);
          float* d = remote(halo, first ? rl : rr) + (unsigned)(2 * p + (first ? 1 : 0)) * nv;
          st4(d + ch0, ld4(c + ch0));  // raw chunks: same layout at both ends
          st4(d + ch1, ld4(c + ch1));
        }
      } else {
        const int q4 = nv / 4;
        if (tid >= T - 2 * q4) {
          const int t = tid - (T - 2 * q4);
          const bool first = t < q4;
          const int ch = first ? t : t - q4;
          float* d = remote(halo, first ? rl : rr) + (unsigned)(2 * p + (first ? 1 : 0)) * nv;
          st4(d + 4 * ch, ld4(col(first ? 0 : n - 1) + 4 * ch));
        }
      }
    }
  };

  // (ii): density and field update (when `update`), then J, P and the
  // sweep constants (when `constants`)
  auto macro_ii = [&](int p, bool update, bool constants) {
    if (w >= nwc) return;
    const float* X = xch(p);
    // neighbour values: left interface (F, m+), right interface (F, m-, rho)
    float Fl = __shfl_up_sync(0xffffffffu, Fc, 1);
    float mpl = __shfl_up_sync(0xffffffffu, mp, 1);
    float Fr = __shfl_down_sync(0xffffffffu, Fc, 1);
    float mmr = __shfl_down_sync(0xffffffffu, mm, 1);
    ff rr_old = ff_shfl_down(rho, 1);
    if (lane == 0) {
      float2 v;
      if (w > 0) v = *reinterpret_cast<const float2*>(wlast + 4 * (p * NW + w - 1));
      else if (C > 1) v = *reinterpret_cast<const float2*>(X);
      else v = *reinterpret_cast<const float2*>(wlast + 4 * (p * NW + nwc - 1));
      Fl = v.x;
      mpl = v.y;
    }
    if (lane == 31) {
      if (w < nwc - 1 || C == 1) {
        const float4 v = ld4(wfirst + 4 * (p * NW + (w < nwc - 1 ? w + 1 : 0)));
        Fr = v.x;
        mmr = v.y;
        rr_old = {v.z, v.w};
      } else {
        const float2 v = *reinterpret_cast<const float2*>(X + 2);
        Fr = v.x;
        mmr = v.y;
        rr_old = ghost;
      }
    }
    ff rho_r = rr_old;
    if (update) {
      // mean flux over the whole state (same order in every thread and CTA)
      float s = 0.f;
      for (int q = lane; q < C * NW; q += 32) s += ((q % NW) < nwc) ? X[4 + q] : 0.f;
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
      const float Fbar = s * f_inv_nx;
      rho = ff_add_f(ff_add_f(rho, Fl), -Fc);
      rho_r = ff_add_f(ff_add_f(rr_old, Fc), -Fr);
      if (C > 1 && tid == n - 1) ghost = rho_r;
      E = ff_add_f(E, -f_dx * (Fc - Fbar));
    }
    if (constants) {
      const float e = E.hi;
      const float dr = (rho_r.hi - rho.hi) + (rho_r.lo - rho.lo);
      const float J = dr * f_inv_dx - e * 0.5f * (rho.hi + rho_r.hi);
      const float ep = e > 0.f ? e : 0.f, em = e < 0.f ? -e : 0.f;
      const float* pe = part + LG * PS + tid;  // end values of the new column
      const float4 en = make_float4(pe[0], pe[PS], pe[2 * PS], pe[3 * PS]);
      const float P = ((mp - mpl) - (mmr - mm)) * f_inv_dx +
                      0.5f * ((ep * en.z - em * en.w) - (ep * en.x - em * en.y));
      st4(par + 4u * (tid + tid / R), make_float4(f_b * ep * f_inv_dv, f_b * em * f_inv_dv, f_b * P, f_b * J));
    }
  };

  // ---------------------------------------------------------------- sweep --
  // registers of the ring: P = old column i-1, Q = i, N = i+1, F = i+2
  float R0[VPT], R1[VPT], R2[VPT], R3[VPT];

  // The neighbouring groups' old columns a sweep needs, by parity p of the
  // step that produced them: the next group's first column (right stash,
  // read at the end of the run, after that group has overwritten it), and,
  // for the first group of a warp, the previous group's last column (left
  // stash: that group belongs to another warp, which may already be
  // sweeping).  Every group writes its entries right after its sweep, before
  // the step's cluster (or block) barrier, which orders them for the
  // readers; the two parities keep the next step's writes off the entries
  // still being read.
  constexpr int GPW = 32 / LG;  // lane groups per warp
  auto stash_r = [&](int p, int gr) { return stash + (unsigned)(p * NGRP + gr) * nv; };
  auto stash_l = [&](int p, int wq) { return stashl + (unsigned)(p * NW + wq) * nv; };
  auto stash_write = [&](int p) {
    const float* c0 = col(i0);
    float* d = stash_r(p, grp == 0 ? NGRP - 1 : grp - 1);
    st4(d + ch0, ld4(c0 + ch0));
    st4(d + ch1, ld4(c0 + ch1));
    const int gn = grp + 1 == NGRP ? 0 : grp + 1;
    if (gn % GPW == 0) {
      const float* cl = col(i0 + R - 1);
      float* e = stash_l(p, gn / GPW);
      st4(e + ch0, ld4(cl + ch0));
      st4(e + ch1, ld4(cl + ch1));
    }
  };
  // old first column of the next group: the right stash, or the right halo
  // for the CTA's last group
  auto right_next = [&](int p) -> const float* {
    if (C > 1 && grp == NGRP - 1) return halo + (unsigned)(2 * p + 1) * nv;
    return stash_r(p, grp);
  };
  // the ring's first columns: the previous group's last column (in this
  // warp: read directly, that group has not started its sweep; else the
  // left stash, or the left halo for the CTA's first group) and this
  // group's first three
  auto preload = [&](int p) {
    const float* lc;
    if (i0 > 0) lc = grp % GPW != 0 ? col(i0 - 1) : stash_l(p, grp / GPW);
    else lc = C > 1 ? halo + (unsigned)(2 * p) * nv : stash_l(p, 0);
    ldcol(R0, lc);
    ldcol(R1, col(i0));
    ldcol(R2, col(i0 + 1));
    ldcol(R3, col(i0 + 2));
  };

  auto sweep = [&](int p) {
    const float* rnext = right_next(p);
    auto body = [&](int k, float (&P)[VPT], float (&Q)[VPT], float (&N)[VPT]) {
      const int i = i0 + k;
      const float4 pr = ld4(par + 4u * (i + grp));  // padded: i / R == grp
      const float ep = pr.x, em = pr.y, bP = pr.z, bJ = pr.w;
      // the v-flux difference -(H_{j+1/2} - H_{j-1/2}) with
      // H_{j+1/2} = ep g_j - em g_{j+1} expands to
      // -(ep + em) g_j + ep g_{j-1} + em g_{j+1}; at the two ends of the
      // velocity grid the outer flux is zero, so node 0 keeps -ep g_0 and
      // node nv-1 keeps -em g_{nv-1}, without the outer neighbour
      const float ae = ep + em;
      float lnb = __shfl_sync(0xffffffffu, Q[VPT - 1], src_left);
      float rnb = __shfl_sync(0xffffffffu, Q[0], src_right);
      if (first_lane) lnb = 0.f;
      if (last_lane) rnb = 0.f;
      const float c0 = first_lane ? ep : ae, c7 = last_lane ? em : ae;
      float out[VPT];
      float ps0 = 0.f, ps1 = 0.f;  // two chains: shorter dependency latency
#pragma unroll
      for (int q = 0; q < VPT; ++q) {
        const float lft = q > 0 ? Q[q > 0 ? q - 1 : 0] : lnb;
        const float rgt = q < VPT - 1 ? Q[q < VPT - 1 ? q + 1 : q] : rnb;
        const float cq = q == 0 ? c0 : (q == VPT - 1 ? c7 : ae);
        const float u = pos ? P[q] : N[q];
        float t = __fmul_rn(bP, Mj[q]);
        t = __fmaf_rn(-bJ, xM[q], t);
        t = __fmaf_rn(al[q], Q[q], t);
        t = __fmaf_rn(be[q], u, t);
        t = __fmaf_rn(-cq, Q[q], t);
        t = __fmaf_rn(ep, lft, t);
        t = __fmaf_rn(em, rgt, t);
        out[q] = t;
        if (q & 1) ps1 = __fmaf_rn(wv[q], t, ps1);
        else ps0 = __fmaf_rn(wv[q], t, ps0);
      }
      stcol(col(i), out);
      put_partial(i, ps0 + ps1, out);
      // bring in old column i + 3 (the next group's, from the stash, at the
      // end of the run) into the slot of column i - 1
      if (k + 3 <= R) ldcol(P, k + 3 < R ? col(i + 3) : rnext);
    };
#pragma unroll
    for (int k = 0; k < R; k += 4) {
      body(k + 0, R0, R1, R2);
      body(k + 1, R1, R2, R3);
      body(k + 2, R2, R3, R0);
      body(k + 3, R3, R0, R1);
    }
  };

  // ------------------------------------------------------------ step loop --
  stash_write(0);  // g^0 (the block barrier after the partials of g^0 made every column visible)
  macro_i(0, false);
  cluster_or_block_sync(C);
  macro_ii(0, false, true);
  preload(0);
  __syncthreads();
  for (int64_t s = 0; s < A.n_steps; ++s) {
    const int pc = (int)(s & 1), pn = pc ^ 1;  // this step's buffers, the next step's
    sweep(pc);
    stash_write(pn);
    // when every group's run is as long as the group is wide, thread t owns
    // cell t, which its own group swept: the partials it sums are the
    // group's (a warp barrier suffices) and the warps run on into macro (i)
    // without waiting for each other
    if (warp_local) __syncwarp();
    else __syncthreads();
    macro_i(pn, true);
    cluster_or_block_sync(C);
    const bool last = s + 1 == A.n_steps;
    macro_ii(pn, true, !last);
    if (!last) preload(pn);
    // when warp-local, everything the next sweep reads from other warps went
    // through the cluster (or block) barrier above; the exit after the last
    // step reads every column
    if (!warp_local || last) __syncthreads();
  }

  // -------------------------------------------------------------- exit ---
  int bad = 0;
  if (has_cell) {
    const double rv = ff_to_double(rho);
    A.rho_out[sbase + a + tid] = rv;
    if (!isfinite(rv)) bad = 1;
    if (A.mask_out) A.mask_out[sbase + a + tid] = 1;
  }
  float* gout = reinterpret_cast<float*>(A.g_buf0) + sbase * nv;
  for (int i = grp; i < n; i += NGRP) {
    float* d = gout + (size_t)(a + i) * nv + VPT * lig;
    *reinterpret_cast<float4*>(d) = ld4(col(i) + ch0);
    *reinterpret_cast<float4*>(d + 4) = ld4(col(i) + ch1);
  }
  if (bad) atomicExch(A.status, (int)MM_ERR_UNSTABLE);
  if (tid == 0 && r == 0 && A.kin_count)
    atomicAdd(A.kin_count, (unsigned long long)A.n_steps * (unsigned long long)nx * (unsigned long long)nv);
}

}  // namespace

// Cluster size and shared-memory bytes of the resident kernel for one state
// shape, or 0 when the shape is not supported (the streaming kernel then
// runs).  Requirements: FP32 g, every cell kinetic, one flux per interface,
// nv = 8 * lanes with lanes in {2, 4, 8, 16, 32}, the cells of a CTA a
// multiple of 32 and at most 256 (one per thread), and runs of a multiple of
// 4 columns for each of the 256 / lanes lane groups.
int fine_resident_cluster(int nx, int nv, bool fp32, bool adapt, int flux_rule, size_t* smem) {
  if (!fp32 || adapt || flux_rule != 0) return 0;
  if (nv % VPT) return 0;
  const int lanes = nv / VPT;
  if (lanes < 2 || lanes > 32 || (lanes & (lanes - 1))) return 0;
  // prefer the smallest cluster whose CTAs fit two to an SM (one CTA's
  // sweep then overlaps the other's latency-bound macro phase), else the
  // smallest that fits at all
  for (const unsigned limit : {115712u, 232448u}) {
    for (int C = 1; C <= 8; C <<= 1) {
      if (nx % C) break;
      const int n = nx / C;
      if (n % 32 || n > T || n % (T / lanes) || (n / (T / lanes)) % 4) continue;
      const unsigned bytes = res_map(n, nv, lanes, C).total;
      if (bytes <= limit) {
        *smem = bytes;
        return C;
      }
    }
  }
  return 0;
}

// Shared-memory bytes of the resident kernel with clusters of C CTAs, or 0
// when that cluster size does not suit the shape (same rules as above, for
// the autotuner).
size_t fine_resident_smem(int nx, int nv, bool fp32, bool adapt, int flux_rule, int C) {
  if (!fp32 || adapt || flux_rule != 0 || nv % VPT) return 0;
  const int lanes = nv / VPT;
  if (lanes < 2 || lanes > 32 || (lanes & (lanes - 1))) return 0;
  if (C < 1 || C > 8 || (C & (C - 1)) || nx % C) return 0;
  const int n = nx / C;
  if (n % 32 || n > T || n % (T / lanes) || (n / (T / lanes)) % 4) return 0;
  const unsigned bytes = res_map(n, nv, lanes, C).total;
  return bytes <= 232448u ? bytes : 0;
}

// Clusters of the resident kernel that the GPU holds at once for this
// launch shape (the occupancy calculator's answer, cached per shape).
template <int LG, int RC, int CC>
static int resident_slots(int C, size_t smem) {
  static std::mutex mu;
  static int dev_c[4] = {-1, -1, -1, -1}, slots_c[4] = {0, 0, 0, 0};
  static size_t smem_c[4] = {0, 0, 0, 0};
  int dev = 0;
  cudaGetDevice(&dev);
  const int ci = C == 1 ? 0 : C == 2 ? 1 : C == 4 ? 2 : 3;
  std::lock_guard<std::mutex> lk(mu);
  if (dev_c[ci] == dev && smem_c[ci] == smem) return slots_c[ci];
  int slots = 0;
  if (C == 1) {
    int per_sm = 0, n_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fine_resident_kernel<LG, RC, CC>, T, smem) == cudaSuccess &&
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      slots = per_sm * n_sm;
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&slots, fine_resident_kernel<LG, RC, CC>, &cfg) != cudaSuccess) slots = 0;
  }
  cudaGetLastError();  // a failed query leaves no sticky error; chunking is then off
  dev_c[ci] = dev;
  smem_c[ci] = smem;
  slots_c[ci] = slots;
  return slots;
}

// Chunks per state of the step range.  With more states than the GPU holds
// at once (Q clusters), one launch of all states runs in ceil(batch / Q)
// waves and the last wave leaves SMs idle (128 states on 74 slots: 2 waves
// for 1.73 waves of work).  Splitting every state's n steps into c chunks of
// n / c steps and running the batch x c items in rounds of Q (chunk-major,
// so a round never holds two chunks of one state and chunk k + 1 of a state
// runs in a later round than chunk k) balances the SMs at the cost of one
// entry and exit per chunk (the state goes through L2 between rounds); the
// n mod c steps left over run as one more chunk of every state.  Every
// launch then has one step count for all its clusters.  Cost model: rounds x
// (chunk + E step-equivalents), with E the entry and exit cost of a chunk:
// measured by mm_autotune on the caller's shape, else kChunkEntry; ties go
// to fewer chunks.
constexpr double kChunkEntry = 8.0;
static double rounds_cost(int batch, int64_t n_steps, int slots, int c, double E) {
  const int64_t L = n_steps / c, r = n_steps % c;
  const int64_t rounds = ((int64_t)batch * c + slots - 1) / slots;
  double cost = (double)rounds * ((double)L + E);
  if (r) cost += (double)((batch + slots - 1) / slots) * ((double)r + E);
  return cost;
}
static int resident_chunks(int batch, int64_t n_steps, int slots, double E) {
  if (slots <= 0 || batch <= slots) return 1;
  if (!(E > 0)) E = kChunkEntry;
  int best = 1;
  double best_cost = rounds_cost(batch, n_steps, slots, 1, E);
  const int cmax = (int)std::min<int64_t>(n_steps, 512);
  for (int c = 2; c <= cmax; ++c) {
    const double q = rounds_cost(batch, n_steps, slots, c, E);
    if (q < 0.99 * best_cost) {
      best = c;
      best_cost = q;
    }
  }
  return best;
}

template <int LG, int RC, int CC>
static cudaError_t configure_res() {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(fine_resident_kernel<LG, RC, CC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  return cudaSuccess;
}

// The launches one call makes: pass 0 runs batch x chunks items of L steps
// in rounds of per_round0 (chunk 0 from the input), pass 1 the r steps left
// over, batch items in rounds of per_round1.
static ResPlan make_plan(int batch, int64_t n_steps, int slots, double E) {
  ResPlan q{};
  q.chunks = resident_chunks(batch, n_steps, slots, E);
  q.L = n_steps / q.chunks;
  q.r = n_steps % q.chunks;
  const int64_t items0 = (int64_t)batch * q.chunks;
  // a round holds at most one chunk of each state
  q.per_round0 = (int)(q.chunks == 1 ? items0 : std::min<int64_t>(slots, batch));
  q.per_round1 = (int)std::min<int64_t>(slots > 0 ? slots : batch, batch);
  q.launches0 = (int)((items0 + q.per_round0 - 1) / q.per_round0);
  q.launches1 = q.r ? (batch + q.per_round1 - 1) / q.per_round1 : 0;
  q.batch = batch;
  return q;
}

int ResPlan::final_launch(int state) const {
  if (r) return launches0 + state / per_round1;
  return (int)(((int64_t)(chunks - 1) * batch + state) / per_round0);
}

template <int LG, int RC, int CC>
static cudaError_t launch_res(FineArgs& a, int C, size_t smem, cudaStream_t s, int* launches,
                              const ResHooks* hooks) {
  cudaError_t e0 = configure_res<LG, RC, CC>();
  if (e0 != cudaSuccess) return e0;
  const ResPlan q = make_plan(a.batch, a.n_steps, resident_slots<LG, RC, CC>(C, smem), a.res_entry_steps);
  const int64_t L = q.L, r = q.r;
  if (launches) *launches = 0;
  int li = 0;  // launch index
  for (int pass = 0; pass < 2; ++pass) {
    const int64_t items = pass == 0 ? (int64_t)a.batch * q.chunks : (r ? a.batch : 0);
    if (items == 0) continue;
    const int64_t per_round = pass == 0 ? q.per_round0 : q.per_round1;
    a.n_steps = pass == 0 ? L : r;
    a.res_from_input = pass == 0 ? 1 : 0;
    for (int64_t i0 = 0; i0 < items; i0 += per_round, ++li) {
      if (hooks && li < ResHooks::kMax && hooks->before[li]) {
        const cudaError_t ew = cudaStreamWaitEvent(s, hooks->before[li], 0);
        if (ew != cudaSuccess) return ew;
      }
      a.res_item0 = (int)i0;
      a.res_state0 = (int)(i0 % a.batch);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(std::min<int64_t>(per_round, items - i0) * C));
      cfg.blockDim = dim3(T);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = C > 1 ? 1 : 0;  // C == 1: a plain launch
      const cudaError_t e = cudaLaunchKernelEx(&cfg, fine_resident_kernel<LG, RC, CC>, (const FineArgs)a, C);
      if (e != cudaSuccess) return e;
      if (launches) ++*launches;
      if (hooks && li < ResHooks::kMax && hooks->after[li]) {
        const cudaError_t er = cudaEventRecord(hooks->after[li], s);
        if (er != cudaSuccess) return er;
      }
    }
  }
  return cudaSuccess;
}

// The run length of a lane group for a shape: the CTA's cells n = nx / C
// over T / LG groups.  The common run of 8 columns has its own unrolled
// instances (with the cluster of 4 fixed too, the batched workload's).
static int run_length(int nx, int nv, int C) { return (nx / C) / (T / (nv / VPT)); }

template <int LG, int RC, int CC>
static int slots_of(int C, size_t smem) {
  if (configure_res<LG, RC, CC>() != cudaSuccess) return 0;
  return resident_slots<LG, RC, CC>(C, smem);
}

template <int LG>
static int plan_slots(int nx, int C, size_t smem) {
  if (run_length(nx, LG * VPT, C) == 8) return C == 4 ? slots_of<LG, 8, 4>(C, smem) : slots_of<LG, 8, 0>(C, smem);
  return slots_of<LG, 0, 0>(C, smem);
}

int resident_capacity(int nx, int nv, int C, size_t smem) {
  switch (nv / VPT) {
    case 2: return plan_slots<2>(nx, C, smem);
    case 4: return plan_slots<4>(nx, C, smem);
    case 8: return plan_slots<8>(nx, C, smem);
    case 16: return plan_slots<16>(nx, C, smem);
    case 32: return plan_slots<32>(nx, C, smem);
  }
  return 0;
}

ResPlan resident_plan(int nx, int nv, int batch, int64_t n_steps, int C, size_t smem, double entry_steps) {
  return make_plan(batch, n_steps, resident_capacity(nx, nv, C, smem), entry_steps);
}

template <int LG>
static cudaError_t launch_lg(FineArgs& a, int C, size_t smem, cudaStream_t s, int* launches, const ResHooks* hooks) {
  if (run_length(a.nx, a.nv, C) == 8) {
    if (C == 4) return launch_res<LG, 8, 4>(a, C, smem, s, launches, hooks);
    return launch_res<LG, 8, 0>(a, C, smem, s, launches, hooks);
  }
  return launch_res<LG, 0, 0>(a, C, smem, s, launches, hooks);
}

cudaError_t launch_fine_resident(const FineArgs& args, int C, size_t smem, cudaStream_t s, int* launches,
                                 const ResHooks* hooks) {
  FineArgs a = args;
  fine_args_floats(a);
  switch (a.nv / VPT) {
    case 2: return launch_lg<2>(a, C, smem, s, launches, hooks);
    case 4: return launch_lg<4>(a, C, smem, s, launches, hooks);
    case 8: return launch_lg<8>(a, C, smem, s, launches, hooks);
    case 16: return launch_lg<16>(a, C, smem, s, launches, hooks);
    case 32: return launch_lg<32>(a, C, smem, s, launches, hooks);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mmk
