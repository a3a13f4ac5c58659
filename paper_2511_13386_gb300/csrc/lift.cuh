// Lifting of order L = 1, 2, 3 (Def. 1, Sec. 3.2-3.3) of one density by one
// thread block, in double: the Chapman-Enskog perturbations of Sec. 2.1
// (eq. Identification) truncated at order L, at the interfaces,
//   g = (I - Pi)[eps h1 + eps^2 h2 + eps^3 h3],
//   h1 = -v M J,  h2 = (v^2 - 1) M K,
//   h3 = v M [dtJ - (v^2 - 1) dK - E (3 - v^2) K],
// K = dJ/dx - E J, dK = dK/dx, dtJ = d2J/dx2 - rho (J - mean J) - E dJ/dx
// (from the drift-diffusion closures d(rho)/dt = dJ/dx, dE/dt = J - mean J),
// with E from the Poisson law, J the S^0 flux, rho at an interface the mean
// of its two cells, and x-derivatives by the Table 1 stencils on the
// interface grid.  The projection uses the discrete moments <v M>,
// <(v^2 - 1) M> = m2 - 1 and <v^3 M> in closed form.
#pragma once
#include <cuda_runtime.h>

namespace mmk {

// Table 1 rows 1 and 2 with integer weights (periodic, unit spacing):
// D1 f = (45 e1 - 9 e2 + e3) / 60, D2 f = (270 s1 - 27 s2 + 2 s3 - 490 f0) / 180,
// e_k = f_{+k} - f_{-k}, s_k = f_{+k} + f_{-k}.
__device__ __forceinline__ int lift_wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ double lift_d1(const double* f, int i, int n) {
  const double e1 = f[lift_wrap(i + 1, n)] - f[lift_wrap(i - 1, n)];
  const double e2 = f[lift_wrap(i + 2, n)] - f[lift_wrap(i - 2, n)];
  const double e3 = f[lift_wrap(i + 3, n)] - f[lift_wrap(i - 3, n)];
  return (45.0 * e1 - 9.0 * e2 + e3) * (1.0 / 60.0);
}

__device__ __forceinline__ double lift_d2(const double* f, int i, int n) {
  const double s1 = f[lift_wrap(i + 1, n)] + f[lift_wrap(i - 1, n)];
  const double s2 = f[lift_wrap(i + 2, n)] + f[lift_wrap(i - 2, n)];
  const double s3 = f[lift_wrap(i + 3, n)] + f[lift_wrap(i - 3, n)];
  return (270.0 * s1 - 27.0 * s2 + 2.0 * s3 - 490.0 * f[i]) * (1.0 / 180.0);
}

// K, dK and dtJ at the interfaces from rho (cells), E and J (interfaces).
// red: >= 32 doubles of shared memory.  Ends with a block barrier.
__device__ inline void lift_fields(const double* rho, const double* E, const double* J, double* K,
                                   double* dK, double* dtJ, int nx, double inv_dx, double* red) {
  const int T = blockDim.x, tid = threadIdx.x;
  double js = 0.0;
  for (int i = tid; i < nx; i += T) {
    dK[i] = lift_d1(J, i, nx) * inv_dx;              // dJ/dx for now
    dtJ[i] = lift_d2(J, i, nx) * (inv_dx * inv_dx);  // d2J/dx2 for now
    js += J[i];
  }
  for (int m = 16; m > 0; m >>= 1) js += __shfl_xor_sync(0xffffffffu, js, m);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = js;
  __syncthreads();
  double Jbar = 0.0;
  for (int q = 0; q < (T >> 5); ++q) Jbar += red[q];
  Jbar /= nx;
  for (int i = tid; i < nx; i += T) {
    const double J1 = dK[i], rho_i = 0.5 * (rho[i] + rho[lift_wrap(i + 1, nx)]);
    K[i] = J1 - E[i] * J[i];
    dtJ[i] = dtJ[i] - rho_i * (J[i] - Jbar) - E[i] * J1;
  }
  __syncthreads();
  for (int i = tid; i < nx; i += T) dK[i] = lift_d1(K, i, nx) * inv_dx;
  __syncthreads();
}

// Lifted g at (interface i, node j with velocity v and Maxwellian M).
struct LiftConsts {
  int L;
  double eps, xiM, m2, mu3;
};

__device__ __forceinline__ double lift_value(const LiftConsts& c, double v, double M, double E, double J, double K,
                                             double dK, double dtJ) {
  const double e = c.eps, v2 = v * v;
  double h = -e * v * M * J;
  double mean = -e * c.xiM * J;
  if (c.L >= 2) {
    h += e * e * (v2 - 1.0) * M * K;
    mean += e * e * (c.m2 - 1.0) * K;
  }
  if (c.L >= 3) {
    const double e3 = e * e * e;
    h += e3 * v * M * (dtJ - (v2 - 1.0) * dK - E * (3.0 - v2) * K);
    mean += e3 * (c.xiM * dtJ - (c.mu3 - c.xiM) * dK - E * (3.0 * c.xiM - c.mu3) * K);
  }
  return h - mean * M;
}

}  // namespace mmk
