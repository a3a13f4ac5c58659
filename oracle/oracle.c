/*
 * Oracle for the space-time hybrid parareal method (Laidin, arXiv 2511.13386).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow, sequential FP64 implementation
 * used to check the CUDA library; only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares nothing with the
 * CUDA path.  Each function cites the passage of the paper it follows.
 *
 * Readings taken where the paper is silent, garbled or self-contradictory
 * (each one is marked "reading:" where it is used):
 *  - Maxwellian exp(-v^2/2), renormalised so that the discrete <M> is 1
 *    (Sec. 1 prints the exponent without its sign).
 *  - Poisson sign as in the schemes S^MM / S^0 / S^HMM:
 *    E_{i+1/2} - E_{i-1/2} = (rho_i - rho_bar) dx; mean-zero gauge for E.
 *  - Upwind fluxes r^+ f_i - r^- f_{i+1} with r^+- = (|r| +- r)/2 >= 0
 *    (Sec. 2.3 prints a "+" between the two terms).
 *  - The projection Pi = <.> M is applied to the whole discrete transport
 *    (x and v parts) so that <g> stays zero with trapezoid weights.
 *  - Trapezoid quadrature on nodes that include +-v_max; the v-transport
 *    treats every node as a width-dv cell with zero flux through the ends.
 *  - Interface status: kinetic iff either adjacent cell is kinetic.
 *  - Kinetic-cell rule, mixed case (one interface norm above the threshold,
 *    the other below): the cell stays kinetic (Sec. 2.2: any one criterion
 *    forces the kinetic description).
 *  - R^eps and R are the same formula (eq. Remainder) on the current rho and
 *    E; the time derivative of E is J - mean(J), from d_x d_t E = d_t rho =
 *    d_x J with the mean-zero gauge.
 *  - Fluxes: one flux per interface (kinetic interface: <xi g>/eps, fluid
 *    interface: -m2 J) so that mass is conserved exactly, as the Remark after
 *    Lemma 1 suggests; flux_rule = 1 keeps the cell-based form printed in
 *    S^HMM, which is not conservative.
 *  - A cell that turns kinetic starts from g = 0 (the fluid state is taken to
 *    be exact equilibrium, Sec. 2.3 last paragraph).
 *  - Algorithm 1 index garbles read as standard parareal
 *    u^{n+1,k+1} = G(u^{n,k+1}) + F(u^{n,k}) - G(u^{n,k}) (Sec. 3.1), with
 *    the loop stopping when k reaches K or the error drops below tol.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- grid -- */

static double dx_of(const orc_params* p) { return p->x_len / p->nx; }
static double dv_of(const orc_params* p) { return 2.0 * p->v_max / (p->nv - 1); }

/* Sec. 2.3 (mesh) and Sec. 1 (Maxwellian); reading: trapezoid weights and a
   discretely normalised Maxwellian. */
double orc_velocity_grid(const orc_params* p, double* v, double* w, double* M) {
  const int nv = p->nv;
  const double dv = dv_of(p);
  for (int j = 0; j < nv; ++j) {
    v[j] = (double)(2 * j - nv + 1) * (0.5 * dv);
    w[j] = (j == 0 || j == nv - 1) ? 0.5 * dv : dv;
  }
  double Z = 0.0;
  for (int j = 0; j < nv; ++j) Z += w[j] * exp(-0.5 * v[j] * v[j]);
  for (int j = 0; j < nv; ++j) M[j] = exp(-0.5 * v[j] * v[j]) / Z;
  double m2 = 0.0;  /* m_2^{dv} of S^0 */
  for (int j = 0; j < nv; ++j) m2 += w[j] * v[j] * v[j] * M[j];
  return m2;
}

/* Table 1, Sec. 2.2: central finite-difference coefficients, offsets -3..3. */
void orc_fd_coefficients(int d, double* c) {
  static const double T[4][7] = {
      {-1.0 / 60, 3.0 / 20, -3.0 / 4, 0.0, 3.0 / 4, -3.0 / 20, 1.0 / 60},
      {1.0 / 90, -3.0 / 20, 3.0 / 2, -49.0 / 18, 3.0 / 2, -3.0 / 20, 1.0 / 90},
      {1.0 / 8, -1.0, 13.0 / 8, 0.0, -13.0 / 8, 1.0, -1.0 / 8},
      {-1.0 / 6, 2.0, -13.0 / 2, 28.0 / 3, -13.0 / 2, 2.0, -1.0 / 6}};
  for (int k = 0; k < 7; ++k) c[k] = T[d - 1][k];
}

static int wrap(int i, int n) { return ((i % n) + n) % n; }

void orc_fd_derivative(int nx, double dx, int d, const double* f, double* out) {
  double c[7];
  orc_fd_coefficients(d, c);
  const double scale = pow(dx, -d);
  for (int i = 0; i < nx; ++i) {
    double s = 0.0;
    for (int k = -3; k <= 3; ++k) s += c[k + 3] * f[wrap(i + k, nx)];
    out[i] = s * scale;
  }
}

/* ------------------------------------------------------------- macro ---- */

/* Discrete Poisson law, last line of S^MM (Sec. 2.3):
   E_{i+1/2} - E_{i-1/2} = (rho_i - rho_bar) dx.  Reading: periodic,
   mean-zero E.  S_i = sum_{m<=i} (rho_m - rho_bar) dx; E = S - mean(S). */
void orc_poisson(const orc_params* p, const double* rho, double* E) {
  const int nx = p->nx;
  const double dx = dx_of(p);
  double S = 0.0, mean = 0.0;
  for (int i = 0; i < nx; ++i) {
    S += (rho[i] - p->rho_bar) * dx;
    E[i] = S;
  }
  for (int i = 0; i < nx; ++i) mean += E[i];
  mean /= nx;
  for (int i = 0; i < nx; ++i) E[i] -= mean;
}

/* Drift-diffusion flux of S^0 (Sec. 2.3): interface density taken as the
   average of the two adjacent cells. */
void orc_flux_J(const orc_params* p, const double* rho, const double* E,
                double* J) {
  const int nx = p->nx;
  const double dx = dx_of(p);
  for (int i = 0; i < nx; ++i) {
    const double r0 = rho[i], r1 = rho[(i + 1) % nx];
    J[i] = (r1 - r0) / dx - E[i] * 0.5 * (r0 + r1);
  }
}

/* L2 norm in velocity of the perturbation at each interface (Sec. 2.2). */
void orc_gnorm(const orc_params* p, const double* g, double* N) {
  const int nx = p->nx, nv = p->nv;
  double* v = malloc(sizeof(double) * nv);
  double* w = malloc(sizeof(double) * nv);
  double* M = malloc(sizeof(double) * nv);
  orc_velocity_grid(p, v, w, M);
  for (int i = 0; i < nx; ++i) {
    double s = 0.0;
    for (int j = 0; j < nv; ++j) s += w[j] * g[(size_t)i * nv + j] * g[(size_t)i * nv + j];
    N[i] = sqrt(s);
  }
  free(v); free(w); free(M);
}

/* Remainder R (eqs. Remainder / RemainderBis, Sec. 2.1) at cell centres with
   the Table 1 differences:
   R = -d3 J + E d2 J + (2 rho - 3 rho_bar) d1 J + 2 J d1 rho - d1 rho d_t E,
   with J = d1 rho - E rho at centres, E_i the average of the two interface
   values and (reading) d_t E = J - mean(J). */
void orc_remainder(const orc_params* p, const double* rho, const double* E,
                   double* R) {
  const int nx = p->nx;
  const double dx = dx_of(p);
  double* Ec = malloc(sizeof(double) * nx);
  double* d1r = malloc(sizeof(double) * nx);
  double* Jc = malloc(sizeof(double) * nx);
  double* d1J = malloc(sizeof(double) * nx);
  double* d2J = malloc(sizeof(double) * nx);
  double* d3J = malloc(sizeof(double) * nx);
  for (int i = 0; i < nx; ++i) Ec[i] = 0.5 * (E[wrap(i - 1, nx)] + E[i]);
  orc_fd_derivative(nx, dx, 1, rho, d1r);
  for (int i = 0; i < nx; ++i) Jc[i] = d1r[i] - Ec[i] * rho[i];
  orc_fd_derivative(nx, dx, 1, Jc, d1J);
  orc_fd_derivative(nx, dx, 2, Jc, d2J);
  orc_fd_derivative(nx, dx, 3, Jc, d3J);
  double meanJ = 0.0;
  for (int i = 0; i < nx; ++i) meanJ += Jc[i];
  meanJ /= nx;
  for (int i = 0; i < nx; ++i) {
    const double dtE = Jc[i] - meanJ;
    R[i] = -d3J[i] + Ec[i] * d2J[i] + (2.0 * rho[i] - 3.0 * p->rho_bar) * d1J[i] +
           2.0 * Jc[i] * d1r[i] - d1r[i] * dtE;
  }
  free(Ec); free(d1r); free(Jc); free(d1J); free(d2J); free(d3J);
}

/* ------------------------------------------------------------ status ---- */

static double r_factor(const orc_params* p) {
  return p->r_scale ? p->eps * p->eps : 1.0;
}

/* Entry status: the kinetic rule of Sec. 2.2 applied as if every cell were
   kinetic, so that F is a pure function of (rho, g). */
void orc_initial_status(const orc_params* p, const double* rho,
                        const double* g, uint8_t* mask) {
  const int nx = p->nx;
  if (!p->adapt) {
    for (int i = 0; i < nx; ++i) mask[i] = 1;
    return;
  }
  double* E = malloc(sizeof(double) * nx);
  double* R = malloc(sizeof(double) * nx);
  double* N = malloc(sizeof(double) * nx);
  orc_poisson(p, rho, E);
  orc_remainder(p, rho, E, R);
  orc_gnorm(p, g, N);
  const double r = r_factor(p);
  for (int i = 0; i < nx; ++i) {
    const double nl = N[wrap(i - 1, nx)], nr = N[i];
    mask[i] = (nl > p->thr_g || nr > p->thr_g || r * fabs(R[i]) > p->thr_R) ? 1 : 0;
  }
  free(E); free(R); free(N);
}

/* Status update of Sec. 2.3 (bullet list after S^HMM):
   fluid cell -> kinetic iff r|R_i| > thr_R;
   kinetic cell -> fluid iff both interface norms <= thr_g and r|R_i| <= thr_R;
   otherwise unchanged. */
void orc_update_status(const orc_params* p, const double* rho,
                       const double* g, uint8_t* mask) {
  const int nx = p->nx;
  if (!p->adapt) return;
  double* E = malloc(sizeof(double) * nx);
  double* R = malloc(sizeof(double) * nx);
  double* N = malloc(sizeof(double) * nx);
  orc_poisson(p, rho, E);
  orc_remainder(p, rho, E, R);
  orc_gnorm(p, g, N);
  const double r = r_factor(p);
  for (int i = 0; i < nx; ++i) {
    const int big_R = r * fabs(R[i]) > p->thr_R;
    if (!mask[i]) {
      mask[i] = big_R ? 1 : 0;
    } else {
      const int small_g = N[wrap(i - 1, nx)] <= p->thr_g && N[i] <= p->thr_g;
      mask[i] = (small_g && !big_R) ? 0 : 1;
    }
  }
  free(E); free(R); free(N);
}

/* ------------------------------------------------------------ dt rule --- */

/* Reading (the paper states no time-step rule): theta times the largest s
   such that, with a = e^{-s/eps^2},
     phi_t = 2 eps (1 - a) v_max / (dx (1 + a))   (upwind transport of g
                                                    with relaxation),
     phi_d = 2 m2 s (1 - a) / dx^2                 (diffusion of rho
                                                    through g),
   (i)   phi_t <= 1,
   (ii)  phi_d <= 1,
   (iv)  phi_d + phi_t / 4 <= 1 (the two couple: the linearised step's
         spectral radius exceeds one near the limit of (ii) once phi_t is
         large; the critical phi_d measured by a von Neumann analysis is
         about 1 - 0.21 phi_t in the diffusive regime),
   (iii) adaptation on: 2 m2 s / dx^2 <= 1 (explicit S^0 in fluid cells),
   the largest s found by bisection. */
static int dt_ok(const orc_params* p, double m2, double s) {
  const double dx = dx_of(p);
  const double a = exp(-s / (p->eps * p->eps));
  const double phi_t = 2.0 * p->eps * (1.0 - a) * p->v_max / (dx * (1.0 + a));
  const double phi_d = 2.0 * m2 * s * (1.0 - a) / (dx * dx);
  if (phi_t > 1.0) return 0;
  if (phi_d > 1.0) return 0;
  if (phi_d + 0.25 * phi_t > 1.0) return 0;
  if (p->adapt && 2.0 * m2 * s / (dx * dx) > 1.0) return 0;
  return 1;
}

double orc_dt_limit(const orc_params* p, double theta) {
  double* v = malloc(sizeof(double) * p->nv);
  double* w = malloc(sizeof(double) * p->nv);
  double* M = malloc(sizeof(double) * p->nv);
  const double m2 = orc_velocity_grid(p, v, w, M);
  free(v); free(w); free(M);
  double lo = 0.0, hi = 1.0;
  while (dt_ok(p, m2, hi)) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (dt_ok(p, m2, mid)) lo = mid; else hi = mid;
  }
  return theta * lo;
}

/* --------------------------------------------------------- fine step ---- */

/* One step of S^HMM (S^MM when every cell is kinetic), Sec. 2.3.
   Reads (rho^n, g^n, s^n), writes (rho^{n+1}, g^{n+1}, s^{n+1}). */
int64_t orc_fine_step(const orc_params* p, double dt, double* rho, double* g,
                      uint8_t* mask) {
  const int nx = p->nx, nv = p->nv;
  const double dx = dx_of(p), dv = dv_of(p), eps = p->eps;
  double* v = malloc(sizeof(double) * nv);
  double* w = malloc(sizeof(double) * nv);
  double* M = malloc(sizeof(double) * nv);
  const double m2 = orc_velocity_grid(p, v, w, M);
  double* E = malloc(sizeof(double) * nx);
  double* J = malloc(sizeof(double) * nx);
  double* Phi = malloc(sizeof(double) * nx);
  uint8_t* kin = malloc(nx);
  uint8_t* cell_kin = malloc(nx);
  double* gn = malloc(sizeof(double) * (size_t)nx * nv);
  double* X = malloc(sizeof(double) * nv);
  memcpy(gn, g, sizeof(double) * (size_t)nx * nv);
  memcpy(cell_kin, mask, nx);

  /* E^n and J^n (S^MM last line; S^0 flux) */
  orc_poisson(p, rho, E);
  orc_flux_J(p, rho, E, J);

  /* interface status under s^n (reading: kinetic iff an adjacent cell is) */
  for (int i = 0; i < nx; ++i) kin[i] = cell_kin[i] || cell_kin[(i + 1) % nx];

  /* status for t^{n+1} from data at t^n (Sec. 2.3) */
  orc_update_status(p, rho, gn, mask);

  const double a = exp(-dt / (eps * eps));
  const double b = eps * (1.0 - a);
  int64_t n_kin = 0;
  for (int i = 0; i < nx; ++i) {
    double* gi = g + (size_t)i * nv;
    if (!kin[i]) {
      /* S^HMM, fluid interface: g^{n+1} = 0 */
      for (int j = 0; j < nv; ++j) gi[j] = 0.0;
      Phi[i] = -m2 * J[i];
      continue;
    }
    ++n_kin;
    const double* gl = gn + (size_t)wrap(i - 1, nx) * nv;
    const double* gc = gn + (size_t)i * nv;
    const double* gr = gn + (size_t)((i + 1) % nx) * nv;
    const double Ei = E[i];
    const double Ep = 0.5 * (fabs(Ei) + Ei), Em = 0.5 * (fabs(Ei) - Ei);
    double P = 0.0;
    for (int j = 0; j < nv; ++j) {
      const double vp = 0.5 * (fabs(v[j]) + v[j]), vm = 0.5 * (fabs(v[j]) - v[j]);
      /* x transport, upwind: (F_{i+1/2} - F_{i-1/2}) / dx */
      const double A = (vp * (gc[j] - gl[j]) - vm * (gr[j] - gc[j])) / dx;
      /* v transport, upwind with zero flux through the ends of the box */
      const double Gr = (j < nv - 1) ? (Ep * gc[j] - Em * gc[j + 1]) : 0.0;
      const double Gl = (j > 0) ? (Ep * gc[j - 1] - Em * gc[j]) : 0.0;
      const double B = (Gr - Gl) / dv;
      X[j] = A + B;
      P += w[j] * X[j];
    }
    /* exponential relaxation of S^MM with the (I - Pi) projection */
    double flux = 0.0;
    for (int j = 0; j < nv; ++j) {
      gi[j] = a * gc[j] - b * (X[j] - P * M[j] + v[j] * M[j] * J[i]);
      flux += w[j] * v[j] * gi[j];
    }
    Phi[i] = flux / eps;
  }

  /* density update: S^HMM with one flux per interface (reading), or the
     cell-based rule as printed when flux_rule == 1 */
  double* rn = malloc(sizeof(double) * nx);
  for (int i = 0; i < nx; ++i) {
    const int il = wrap(i - 1, nx);
    double fr = Phi[i], fl = Phi[il];
    if (p->flux_rule == 1) {
      if (cell_kin[i]) {
        fr = kin[i] ? Phi[i] : 0.0;
        fl = kin[il] ? Phi[il] : 0.0;
      } else {
        fr = -m2 * J[i];
        fl = -m2 * J[il];
      }
    }
    rn[i] = rho[i] - dt / dx * (fr - fl);
  }
  memcpy(rho, rn, sizeof(double) * nx);

  free(rn); free(v); free(w); free(M); free(E); free(J); free(Phi);
  free(kin); free(cell_kin); free(gn); free(X);
  return n_kin;
}

void orc_fine(const orc_params* p, int64_t n_steps, double dt, double* rho,
              double* g, uint8_t* mask_out, orc_fine_stats* stats) {
  uint8_t* mask = malloc(p->nx);
  orc_initial_status(p, rho, g, mask);
  int64_t kin_updates = 0;
  for (int64_t s = 0; s < n_steps; ++s)
    kin_updates += orc_fine_step(p, dt, rho, g, mask) * p->nv;
  if (mask_out) memcpy(mask_out, mask, p->nx);
  if (stats) {
    stats->steps = n_steps;
    stats->kinetic_updates = kin_updates;
  }
  free(mask);
}

/* ----------------------------------------------------------- coarse ----- */

/* One explicit step of the limit scheme S^0 (Sec. 2.3). */
void orc_limit_step(const orc_params* p, double dt, double* rho) {
  const int nx = p->nx;
  const double dx = dx_of(p);
  double* v = malloc(sizeof(double) * p->nv);
  double* w = malloc(sizeof(double) * p->nv);
  double* M = malloc(sizeof(double) * p->nv);
  const double m2 = orc_velocity_grid(p, v, w, M);
  double* E = malloc(sizeof(double) * nx);
  double* J = malloc(sizeof(double) * nx);
  double* rn = malloc(sizeof(double) * nx);
  orc_poisson(p, rho, E);
  orc_flux_J(p, rho, E, J);
  for (int i = 0; i < nx; ++i)
    rn[i] = rho[i] + m2 * dt / dx * (J[i] - J[wrap(i - 1, nx)]);
  memcpy(rho, rn, sizeof(double) * nx);
  free(v); free(w); free(M); free(E); free(J); free(rn);
}

/* Cyclic tridiagonal solve, Sherman-Morrison on top of the Thomas
   algorithm: lo[i] x[i-1] + di[i] x[i] + up[i] x[i+1] = r[i], indices
   periodic.  Overwrites r with x. */
static void cyclic_tridiag(int n, const double* lo, const double* di,
                           const double* up, double* r) {
  double* bb = malloc(sizeof(double) * n);
  double* u = malloc(sizeof(double) * n);
  double* c = malloc(sizeof(double) * n);
  double* z = malloc(sizeof(double) * n);
  const double alpha = up[n - 1]; /* A[n-1][0] */
  const double beta = lo[0];      /* A[0][n-1] */
  const double gamma = -di[0];
  for (int i = 0; i < n; ++i) bb[i] = di[i];
  bb[0] = di[0] - gamma;
  bb[n - 1] = di[n - 1] - alpha * beta / gamma;
  for (int i = 0; i < n; ++i) u[i] = 0.0;
  u[0] = gamma;
  u[n - 1] = alpha;
  /* Thomas on (lo, bb, up) for r and for u */
  double* rhs[2] = {r, u};
  double* out[2] = {r, z};
  for (int k = 0; k < 2; ++k) {
    double* x = out[k];
    const double* d = rhs[k];
    double bet = bb[0];
    x[0] = d[0] / bet;
    for (int i = 1; i < n; ++i) {
      c[i] = up[i - 1] / bet;
      bet = bb[i] - lo[i] * c[i];
      x[i] = (d[i] - lo[i] * x[i - 1]) / bet;
    }
    for (int i = n - 2; i >= 0; --i) x[i] -= c[i + 1] * x[i + 1];
  }
  const double fact = (r[0] + beta * r[n - 1] / gamma) /
                      (1.0 + z[0] + beta * z[n - 1] / gamma);
  for (int i = 0; i < n; ++i) r[i] -= fact * z[i];
  free(bb); free(u); free(c); free(z);
}

/* Linearly implicit S^0 step (reading; "1 step per slice" for G):
   E frozen from rho^m, then (I - m2 dt L) rho^{m+1} = rho^m with
   (L rho)_i = (J_{i+1/2} - J_{i-1/2}) / dx and J as in S^0. */
void orc_limit_step_implicit(const orc_params* p, double dt, double* rho) {
  const int nx = p->nx;
  const double dx = dx_of(p);
  double* v = malloc(sizeof(double) * p->nv);
  double* w = malloc(sizeof(double) * p->nv);
  double* M = malloc(sizeof(double) * p->nv);
  const double m2 = orc_velocity_grid(p, v, w, M);
  double* E = malloc(sizeof(double) * nx);
  double* lo = malloc(sizeof(double) * nx);
  double* di = malloc(sizeof(double) * nx);
  double* up = malloc(sizeof(double) * nx);
  orc_poisson(p, rho, E);
  const double k = m2 * dt / dx;
  for (int i = 0; i < nx; ++i) {
    const double Er = E[i], El = E[wrap(i - 1, nx)];
    /* coefficients of L (times dx) on rho_{i-1}, rho_i, rho_{i+1} */
    const double cl = 1.0 / dx + 0.5 * El;
    const double cc = -2.0 / dx - 0.5 * Er + 0.5 * El;
    const double cr = 1.0 / dx - 0.5 * Er;
    lo[i] = -k * cl;
    di[i] = 1.0 - k * cc;
    up[i] = -k * cr;
  }
  cyclic_tridiag(nx, lo, di, up, rho);
  free(v); free(w); free(M); free(E); free(lo); free(di); free(up);
}

void orc_coarse(const orc_params* p, int kind, int n_sub, double t_span,
                double* rho) {
  const double dt = t_span / n_sub;
  for (int s = 0; s < n_sub; ++s) {
    if (kind == 0) orc_limit_step_implicit(p, dt, rho);
    else orc_limit_step(p, dt, rho);
  }
}

/* ------------------------------------------------------------- lift ----- */

/* Lifting of order one (Def. 1 with L = 1 and the identification
   h^(1) = -T(rho M), Sec. 2.1 / 3.3): at interfaces, with the interface
   density averaged (Sec. 3.3),  g = -eps (I - Pi)[xi M J]. */
void orc_lift(const orc_params* p, const double* rho, double* g) {
  const int nx = p->nx, nv = p->nv;
  double* v = malloc(sizeof(double) * nv);
  double* w = malloc(sizeof(double) * nv);
  double* M = malloc(sizeof(double) * nv);
  orc_velocity_grid(p, v, w, M);
  double* E = malloc(sizeof(double) * nx);
  double* J = malloc(sizeof(double) * nx);
  orc_poisson(p, rho, E);
  orc_flux_J(p, rho, E, J);
  double xiM = 0.0;  /* <xi M> */
  for (int j = 0; j < nv; ++j) xiM += w[j] * v[j] * M[j];
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < nv; ++j)
      g[(size_t)i * nv + j] = -p->eps * (v[j] * M[j] * J[i] - xiM * J[i] * M[j]);
  free(v); free(w); free(M); free(E); free(J);
}

/* Lifting of order L (Def. 1): the Chapman-Enskog perturbations h1..hL of
   the identification in Sec. 2.1 evaluated at the interfaces, summed with
   weights eps^l, then projected with (I - Pi) so that <g> = 0 exactly.
   h2 and h3 follow from h^{(l+1)} = -dt h^{(l-1)} - T h^{(l)} with
   T f = v df/dx + E df/dv, dv M = -v M, and the drift-diffusion closures
   d(rho)/dt = dJ/dx, dE/dt = J - mean J:
     h2 = (v^2 - 1) M (dJ/dx - E J)
     h3 = v M [dJ/dt - (v^2 - 1) dK/dx - E (3 - v^2) K],  K = dJ/dx - E J,
     dJ/dt = d2J/dx2 - rho (J - mean J) - E dJ/dx. */
void orc_lift_order(const orc_params* p, int L, const double* rho, double* g) {
  const int nx = p->nx, nv = p->nv;
  const double dx = p->x_len / nx, eps = p->eps;
  double* v = malloc(sizeof(double) * nv);
  double* w = malloc(sizeof(double) * nv);
  double* M = malloc(sizeof(double) * nv);
  orc_velocity_grid(p, v, w, M);
  double* E = malloc(sizeof(double) * nx);
  double* J = malloc(sizeof(double) * nx);
  double* J1 = malloc(sizeof(double) * nx);  /* dJ/dx */
  double* J2 = malloc(sizeof(double) * nx);  /* d2J/dx2 */
  double* K = malloc(sizeof(double) * nx);
  double* K1 = malloc(sizeof(double) * nx);  /* dK/dx */
  double* h = malloc(sizeof(double) * nv);
  orc_poisson(p, rho, E);
  orc_flux_J(p, rho, E, J);
  orc_fd_derivative(nx, dx, 1, J, J1);
  orc_fd_derivative(nx, dx, 2, J, J2);
  for (int i = 0; i < nx; ++i) K[i] = J1[i] - E[i] * J[i];
  orc_fd_derivative(nx, dx, 1, K, K1);
  double Jbar = 0.0;
  for (int i = 0; i < nx; ++i) Jbar += J[i];
  Jbar /= nx;
  for (int i = 0; i < nx; ++i) {
    const double rho_i = 0.5 * (rho[i] + rho[(i + 1) % nx]);
    const double dtJ = J2[i] - rho_i * (J[i] - Jbar) - E[i] * J1[i];
    double mean = 0.0;
    for (int j = 0; j < nv; ++j) {
      const double v2 = v[j] * v[j];
      double hj = eps * (-v[j] * M[j] * J[i]);
      if (L >= 2) hj += eps * eps * (v2 - 1.0) * M[j] * K[i];
      if (L >= 3)
        hj += eps * eps * eps * v[j] * M[j] * (dtJ - (v2 - 1.0) * K1[i] - E[i] * (3.0 - v2) * K[i]);
      h[j] = hj;
      mean += w[j] * hj;
    }
    for (int j = 0; j < nv; ++j) g[(size_t)i * nv + j] = h[j] - mean * M[j];
  }
  free(v); free(w); free(M); free(E); free(J); free(J1); free(J2); free(K); free(K1); free(h);
}

static void relift(const orc_params* p, const orc_parareal_cfg* c, const double* rho, double* g) {
  if (c->lift_order > 1) orc_lift_order(p, c->lift_order, rho, g);
  else orc_lift(p, rho, g);
}

/* ---------------------------------------------------------- parareal ---- */

static int64_t steps_for(double span, double dt_lim) {
  int64_t n = (int64_t)ceil(span / dt_lim);
  return n < 1 ? 1 : n;
}

/* Algorithm 1 (Sec. 3.3) in the standard parareal reading of Sec. 3.1.
   The correction is evaluated as F + (G_new - G_old), which equals the
   printed G_new + F - G_old and is exact (bitwise F) on converged slices. */
/* Algorithm 1 on the full micro-macro state U = (rho, g): F(U) is S^HMM
   from the slice's own (rho, g) (no relifting), G(U) = (G rho, L G rho)
   (the coarse density and its lifting), and the correction
   U^{n+1,k+1} = F(U^{n,k}) + (G(U^{n,k+1}) - G(U^{n,k})) acts on both parts
   (Sec. 3.1 applied to the state of the fine scheme).  Converged slices
   equal the plain sequential F, without relifting.  The successive error is
   measured on the density. */
static int parareal_full(const orc_params* p, const orc_parareal_cfg* c,
                         const double* rho0, const double* g0, double* rho_slices,
                         double* err) {
  const int nx = p->nx, nv = p->nv, N = c->n_slices;
  const size_t G1 = (size_t)nx * nv;
  const double span = c->t_end / N;
  const int64_t nf = steps_for(span, c->dt_fine);
  const double dtf = span / nf;
  double* Gprev = malloc(sizeof(double) * (size_t)(N + 1) * nx);
  double* Frho = malloc(sizeof(double) * (size_t)(N + 1) * nx);
  double* Fg = malloc(sizeof(double) * (size_t)(N + 1) * G1);
  double* next = malloc(sizeof(double) * (size_t)(N + 1) * nx);
  double* gs = malloc(sizeof(double) * (size_t)(N + 1) * G1);     /* g^{n,k} */
  double* gnext = malloc(sizeof(double) * (size_t)(N + 1) * G1);
  double* tmp = malloc(sizeof(double) * nx);
  double* lnew = malloc(sizeof(double) * G1);
  double* lold = malloc(sizeof(double) * G1);

  /* coarse guess U^{n+1,0} = G(U^{n,0}) */
  memcpy(rho_slices, rho0, sizeof(double) * nx);
  memcpy(gs, g0, sizeof(double) * G1);
  for (int n = 0; n < N; ++n) {
    memcpy(tmp, rho_slices + (size_t)n * nx, sizeof(double) * nx);
    orc_coarse(p, c->coarse_kind, c->coarse_steps, span, tmp);
    memcpy(rho_slices + (size_t)(n + 1) * nx, tmp, sizeof(double) * nx);
    memcpy(Gprev + (size_t)(n + 1) * nx, tmp, sizeof(double) * nx);
    relift(p, c, tmp, gs + (size_t)(n + 1) * G1);
  }

  int k = 0;
  for (; k < c->max_iter && k < N; ++k) {
    for (int n = k; n < N; ++n) {  /* F(U^{n,k}) */
      double* r = Frho + (size_t)(n + 1) * nx;
      double* g = Fg + (size_t)(n + 1) * G1;
      memcpy(r, rho_slices + (size_t)n * nx, sizeof(double) * nx);
      memcpy(g, gs + (size_t)n * G1, sizeof(double) * G1);
      orc_fine(p, nf, dtf, r, g, NULL, NULL);
    }
    memcpy(next, rho_slices, sizeof(double) * (size_t)(k + 1) * nx);
    memcpy(gnext, gs, sizeof(double) * (size_t)(k + 1) * G1);
    for (int n = k; n < N; ++n) {
      memcpy(tmp, next + (size_t)n * nx, sizeof(double) * nx);
      orc_coarse(p, c->coarse_kind, c->coarse_steps, span, tmp);
      double* out = next + (size_t)(n + 1) * nx;
      const double* F = Frho + (size_t)(n + 1) * nx;
      const double* Go = Gprev + (size_t)(n + 1) * nx;
      for (int i = 0; i < nx; ++i) out[i] = F[i] + (tmp[i] - Go[i]);
      relift(p, c, tmp, lnew);
      relift(p, c, Go, lold);
      double* gout = gnext + (size_t)(n + 1) * G1;
      const double* FG = Fg + (size_t)(n + 1) * G1;
      for (size_t q = 0; q < G1; ++q) gout[q] = FG[q] + (lnew[q] - lold[q]);
      memcpy(Gprev + (size_t)(n + 1) * nx, tmp, sizeof(double) * nx);
    }
    double e = 0.0;
    for (size_t q = 0; q < (size_t)(N + 1) * nx; ++q) {
      const double d = fabs(next[q] - rho_slices[q]);
      if (d > e) e = d;
    }
    memcpy(rho_slices, next, sizeof(double) * (size_t)(N + 1) * nx);
    memcpy(gs, gnext, sizeof(double) * (size_t)(N + 1) * G1);
    if (err) err[k] = e;
    if (e < c->tol) { ++k; break; }
  }
  free(Gprev); free(Frho); free(Fg); free(next); free(gs); free(gnext); free(tmp); free(lnew); free(lold);
  return k;
}

int orc_parareal(const orc_params* p, const orc_parareal_cfg* c,
                 const double* rho0, const double* g0, double* rho_slices,
                 double* err) {
  if (c->mode == 1) return parareal_full(p, c, rho0, g0, rho_slices, err);
  const int nx = p->nx, nv = p->nv, N = c->n_slices;
  const double span = c->t_end / N;
  const int64_t nf = steps_for(span, c->dt_fine);
  const double dtf = span / nf;
  double* Gprev = malloc(sizeof(double) * (size_t)(N + 1) * nx);
  double* Frho = malloc(sizeof(double) * (size_t)(N + 1) * nx);
  double* next = malloc(sizeof(double) * (size_t)(N + 1) * nx);
  double* g = malloc(sizeof(double) * (size_t)nx * nv);
  double* tmp = malloc(sizeof(double) * nx);

  /* first coarse guess of Algorithm 1 */
  memcpy(rho_slices, rho0, sizeof(double) * nx);
  for (int n = 0; n < N; ++n) {
    memcpy(tmp, rho_slices + (size_t)n * nx, sizeof(double) * nx);
    orc_coarse(p, c->coarse_kind, c->coarse_steps, span, tmp);
    memcpy(rho_slices + (size_t)(n + 1) * nx, tmp, sizeof(double) * nx);
    memcpy(Gprev + (size_t)(n + 1) * nx, tmp, sizeof(double) * nx);
  }

  int k = 0;
  for (; k < c->max_iter && k < N; ++k) {
    /* fine propagations from (rho^{n,k}, L rho^{n,k}), n = k..N-1 */
    for (int n = k; n < N; ++n) {
      double* r = Frho + (size_t)(n + 1) * nx;
      memcpy(r, rho_slices + (size_t)n * nx, sizeof(double) * nx);
      if (n == 0) memcpy(g, g0, sizeof(double) * (size_t)nx * nv);
      else relift(p, c, r, g);
      orc_fine(p, nf, dtf, r, g, NULL, NULL);
    }
    /* sequential correction */
    memcpy(next, rho_slices, sizeof(double) * (size_t)(k + 1) * nx);
    for (int n = k; n < N; ++n) {
      memcpy(tmp, next + (size_t)n * nx, sizeof(double) * nx);
      orc_coarse(p, c->coarse_kind, c->coarse_steps, span, tmp);
      double* out = next + (size_t)(n + 1) * nx;
      const double* F = Frho + (size_t)(n + 1) * nx;
      const double* Go = Gprev + (size_t)(n + 1) * nx;
      for (int i = 0; i < nx; ++i) out[i] = F[i] + (tmp[i] - Go[i]);
      memcpy(Gprev + (size_t)(n + 1) * nx, tmp, sizeof(double) * nx);
    }
    double e = 0.0;
    for (size_t q = 0; q < (size_t)(N + 1) * nx; ++q) {
      const double d = fabs(next[q] - rho_slices[q]);
      if (d > e) e = d;
    }
    memcpy(rho_slices, next, sizeof(double) * (size_t)(N + 1) * nx);
    if (err) err[k] = e;
    if (e < c->tol) { ++k; break; }
  }
  free(Gprev); free(Frho); free(next); free(g); free(tmp);
  return k;
}

void orc_sequential(const orc_params* p, const orc_parareal_cfg* c,
                    const double* rho0, const double* g0, double* rho_slices) {
  const int nx = p->nx, nv = p->nv, N = c->n_slices;
  const double span = c->t_end / N;
  const int64_t nf = steps_for(span, c->dt_fine);
  const double dtf = span / nf;
  double* g = malloc(sizeof(double) * (size_t)nx * nv);
  memcpy(rho_slices, rho0, sizeof(double) * nx);
  for (int n = 0; n < N; ++n) {
    double* r = rho_slices + (size_t)(n + 1) * nx;
    memcpy(r, rho_slices + (size_t)n * nx, sizeof(double) * nx);
    if (n == 0) memcpy(g, g0, sizeof(double) * (size_t)nx * nv);
    else if (c->mode != 1) relift(p, c, r, g);  /* full state: g carried on */
    orc_fine(p, nf, dtf, r, g, NULL, NULL);
  }
  free(g);
}
