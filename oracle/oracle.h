/*
 * Oracle for the space-time hybrid parareal method (Laidin, arXiv 2511.13386).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, sequential FP64 C
 * implementation of what the GPU library computes.  It exists to check the
 * CUDA path; only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or constant
 * with the CUDA library.
 *
 * Discretisation (1D-1V, Sec. 2.3; the paper's experiments use d_v = 3, this
 * oracle uses one velocity dimension):
 *   x in [0, x_len) periodic, Nx cells X_i, dx = x_len / Nx.  Cell data
 *   (rho, status, remainder R) at centres; interface data (g, E, J, flux)
 *   at x_{i+1/2}, stored at index i.
 *   v_j = (2j - Nv + 1) dv / 2 on [-v_max, v_max], dv = 2 v_max / (Nv - 1),
 *   trapezoid weights w_j (dv, halved at both ends); <h> = sum_j w_j h_j.
 *   M_j = exp(-v_j^2/2) / Z with Z chosen so that <M> = 1 (the Maxwellian of
 *   Sec. 1 with the sign of the exponent taken as negative).
 *
 * Arrays: rho[nx], g[nx][nv] (v contiguous), E[nx], J[nx], mask[nx] (1 =
 * kinetic cell).  Every function is a pure function of its arguments.
 *
 * Parity unpinned (no closed form or printed value fixes it; any consistent
 * choice passes): the discrete time derivative of E inside R.  Which
 * scaling of the remainder criterion the paper means (literal |R| or
 * eps^2 |R|) is a reading, but each switch is pinned, as is the cell-based
 * density update (flux_rule = 1).  The lifting of orders two and three is
 * pinned to its continuous limit and to the scheme's own relaxed
 * perturbation, not to a printed value.
 */
#ifndef ORACLE_H
#define ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t nx, nv;
  double x_len;     /* torus length (1.0 in every workload) */
  double v_max;     /* velocity box [-v_max, v_max] */
  double eps;       /* Knudsen number */
  double rho_bar;   /* neutralising background density of the Poisson law */
  int32_t adapt;    /* 0: every cell kinetic (S^MM); 1: hybrid S^HMM */
  double thr_g;     /* threshold on ||g||_2 at an interface */
  double thr_R;     /* threshold on the macroscopic remainder */
  int32_t r_scale;  /* 0: compare |R| (literal); 1: compare eps^2 |R| */
  int32_t flux_rule;/* 0: one flux per interface (conservative);
                       1: cell-based rule as printed in S^HMM */
} orc_params;

/* velocity grid: v, w, M (each nv long); returns m2 = <v^2 M> */
double orc_velocity_grid(const orc_params* p, double* v, double* w, double* M);

/* Table 1 (Sec. 2.2): 7-point central coefficients of derivative order
   d = 1..4, offsets -3..3; coef must hold 7 doubles. */
void orc_fd_coefficients(int d, double* coef);

/* periodic finite-difference derivative of order d with Table 1 */
void orc_fd_derivative(int nx, double dx, int d, const double* f, double* out);

/* discrete Poisson law of S^MM: E_{i+1/2}-E_{i-1/2} = (rho_i - rho_bar) dx,
   periodic, mean-zero gauge */
void orc_poisson(const orc_params* p, const double* rho, double* E);

/* drift-diffusion flux of S^0: J_{i+1/2} = (rho_{i+1}-rho_i)/dx
   - E_{i+1/2} (rho_i + rho_{i+1})/2 */
void orc_flux_J(const orc_params* p, const double* rho, const double* E,
                double* J);

/* interface norms N_{i+1/2} = sqrt(<g_{i+1/2}^2>) */
void orc_gnorm(const orc_params* p, const double* g, double* N);

/* macroscopic remainder R_i (eq. Remainder, Sec. 2.1) with Table 1 */
void orc_remainder(const orc_params* p, const double* rho, const double* E,
                   double* R);

/* status at F entry: kinetic iff either adjacent interface norm > thr_g or
   r|R| > thr_R (every cell kinetic when adapt == 0) */
void orc_initial_status(const orc_params* p, const double* rho,
                        const double* g, uint8_t* mask);

/* status update of Sec. 2.3 from data at t^n (mask in: s^n, out: s^{n+1}) */
void orc_update_status(const orc_params* p, const double* rho,
                       const double* g, uint8_t* mask);

/* Time-step rule: theta times the largest s meeting the stability
   conditions, found by bisection.  Returns the step limit. */
double orc_dt_limit(const orc_params* p, double theta);

/* one step of S^HMM (S^MM when every cell is kinetic); rho, g and mask
   are updated in place; returns the number of kinetic interfaces */
int64_t orc_fine_step(const orc_params* p, double dt, double* rho, double* g,
                      uint8_t* mask);

typedef struct {
  int64_t steps;            /* time steps taken */
  int64_t kinetic_updates;  /* sum over steps of kinetic interfaces * nv */
} orc_fine_stats;

/* F: n_steps steps of S^HMM from (rho, g) with the entry status; in place;
   mask_out (nullable) receives the final status */
void orc_fine(const orc_params* p, int64_t n_steps, double dt, double* rho,
              double* g, uint8_t* mask_out, orc_fine_stats* stats);

/* one explicit S^0 step */
void orc_limit_step(const orc_params* p, double dt, double* rho);

/* one linearly implicit S^0 step: E frozen from rho, then
   (I - m2 dt L_E) rho_new = rho solved as a cyclic tridiagonal system */
void orc_limit_step_implicit(const orc_params* p, double dt, double* rho);

/* G over a span: kind 0 = implicit with n_sub equal steps,
   kind 1 = explicit with n_sub equal steps */
void orc_coarse(const orc_params* p, int kind, int n_sub, double t_span,
                double* rho);

/* lifting of order one (Def. 1, Sec. 3.2-3.3):
   g_{i+1/2,j} = -eps (I - Pi)[xi_j M_j J_{i+1/2}] */
void orc_lift(const orc_params* p, const double* rho, double* g);

/* lifting of order L = 1, 2, 3 (Def. 1 with the identification of Sec. 2.1,
   eq. Identification, truncated at L; d_x = d_v = 1):
     g = (I - Pi)[eps h1 + eps^2 h2 + eps^3 h3]   (terms up to order L)
     h1_j = -v_j M_j J
     h2_j = (v_j^2 - 1) M_j K,                      K = dJ/dx - E J
     h3_j = v_j M_j [dJ/dt - (v_j^2 - 1) dK/dx - E (3 - v_j^2) K]
   with dtJ = d2J/dx2 - rho (J - mean J) - E dJ/dx (the drift-diffusion
   closures d(rho)/dt = dJ/dx and dE/dt = J - mean J).  Everything lives at
   the interfaces: E from the Poisson law, J the S^0 flux, rho the mean of
   the two neighbouring cells (Sec. 3.3 uses interface averages of the
   density); x-derivatives are the Table 1 stencils on the interface grid.
   L = 1 is orc_lift. */
void orc_lift_order(const orc_params* p, int L, const double* rho, double* g);

typedef struct {
  double t_end;       /* T */
  int32_t n_slices;   /* N_g */
  int32_t max_iter;   /* K */
  double tol;         /* stop when the successive error is below tol */
  int32_t coarse_kind, coarse_steps;
  double dt_fine;     /* fine step limit; per slice n = ceil(slice/dt_fine) */
  int32_t lift_order; /* L of the relifting (0 or 1: order one) */
  int32_t mode;       /* 0: density only, relifted at every slice (Alg. 1);
                         1: full state (rho, g), G(U) = (G rho, L G rho) */
} orc_parareal_cfg;

/* Algorithm 1 (Sec. 3.3): rho-only parareal with relifting.
   rho_slices: (N+1) x nx output; err: max_iter successive errors.
   Returns the number of iterations performed. */
int orc_parareal(const orc_params* p, const orc_parareal_cfg* c,
                 const double* rho0, const double* g0, double* rho_slices,
                 double* err);

/* sequential fine reference of the same problem: rho^{n+1} =
   F_rho(rho^n, L rho^n) (g0 for the first slice), with the lifting of
   order c->lift_order; with c->mode == 1, the plain F carried through the
   slices without relifting */
void orc_sequential(const orc_params* p, const orc_parareal_cfg* c,
                    const double* rho0, const double* g0, double* rho_slices);

#ifdef __cplusplus
}
#endif
#endif
