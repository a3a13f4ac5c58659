/*
 * mm.h -- C ABI of the GB300 hybrid micro-macro parareal library (libmm).
 *
 * The library implements, on one GB300 GPU (sm_103a), the hot path of the
 * space-time hybrid parareal method for the 1D-1V linear Vlasov-Poisson-BGK
 * equation in the diffusive scaling (T. Laidin, arXiv 2511.13386):
 *   - the fine propagator F = S^HMM, the spatially hybridised micro-macro
 *     asymptotic-preserving scheme (Sec. 2.3, eqs. S^MM and S^HMM), run for a
 *     whole batch of parareal slice states in one launch;
 *   - the coarse propagator G = S^0 (Sec. 2.3, eq. S^0), the lifting of
 *     Def. 1 (Sec. 3.2-3.3) and the parareal loop of Algorithm 1 (Sec. 3.3),
 *     kept on the device beside F.
 *
 * Discretisation (shared by every entry point):
 *   x in [0, x_len) periodic, nx cells, dx = x_len / nx.  Cell data (rho,
 *   status) at cell centres x_i = (i + 1/2) dx; interface data (g, E, J) at
 *   x_{i+1/2} = (i + 1) dx, stored at index i.
 *   v_j = (2j - nv + 1) dv / 2 on [-v_max, v_max], dv = 2 v_max / (nv - 1);
 *   trapezoid weights; Maxwellian exp(-v^2/2) normalised so that its
 *   discrete integral is one.
 *
 * Array layouts (row-major, C order):
 *   rho  : double [batch][nx]
 *   g    : [batch][nx][nv], v contiguous; double for MM_FP64, float for
 *          MM_FP32G
 *   mask : uint8_t [batch][nx], 1 = kinetic cell, 0 = fluid cell
 *
 * Pointers: every array argument may be a device pointer (the fast path) or
 * a host pointer (pageable or pinned); host arrays are staged through device
 * memory inside the call, on the call's stream.  The caller owns every
 * array it passes.  The library owns its workspace, obtained through the
 * optional mm_alloc callbacks (default: cudaMallocAsync on the call's
 * stream) and released by mm_destroy.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).  Device-pointer calls are asynchronous on that stream
 * unless a stats pointer is given, in which case the call synchronises the
 * stream before returning.
 *
 * Errors: every call returns an mm_status; the message of the last failure
 * on the calling thread is available from mm_last_error().  Arguments are
 * validated before anything is launched.  No call aborts or throws.
 *
 * Threads: an mm_ctx is not thread-safe (one thread at a time); an
 * mm_server is thread-safe for serve_submit / serve_poll.
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MM_ABI_VERSION 1

/* Exported symbols (the library is built with hidden default visibility). */
#if defined(MM_BUILD) && defined(__GNUC__)
#define MM_API __attribute__((visibility("default")))
#else
#define MM_API
#endif

typedef enum {
  MM_OK = 0,
  MM_ERR_INVALID = 1,         /* bad argument, size or parameter */
  MM_ERR_OOM = 2,             /* device allocation failed */
  MM_ERR_CUDA = 3,            /* a CUDA runtime call failed */
  MM_ERR_TIMEOUT = 4,         /* a bounded wait ran out */
  MM_ERR_UNSTABLE = 5,        /* step above the stability limit, or a
                                 non-finite density was produced */
  MM_ERR_BUSY = 6,            /* server at capacity (admission refused) */
  MM_ERR_NOT_READY = 7,       /* result not ready before the poll timeout */
  MM_ERR_UNKNOWN_TICKET = 8   /* no such request */
} mm_status;

typedef enum {
  MM_FP64 = 0,   /* g stored and updated in double; every sum in double */
  MM_FP32G = 1   /* g stored and updated in float, its velocity moments
                    summed in float; density, field (Poisson law), fluid
                    flux and the criteria's stencils in float-float (~48-bit)
                    arithmetic, so mass is kept to float-float rounding;
                    output density double */
} mm_precision;

/* Optional device-memory callbacks (e.g. a framework's caching allocator). */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, void* stream, void* user);
  void* user;
} mm_alloc;

/* Problem description.  Fill with mm_params_default() then override. */
typedef struct {
  int32_t nx;          /* cells, 8 <= nx <= 65536 */
  int32_t nv;          /* velocity nodes: even, >= 4, see mm_params_default */
  double x_len;        /* torus length (> 0) */
  double v_max;        /* velocity box half-width (> 0) */
  double eps;          /* Knudsen number (> 0) */
  double rho_bar;      /* neutralising density of the Poisson law
                          (Sec. 1, eq. Poisson); NaN = the mean of each
                          input density */
  int32_t adapt;       /* 0: every cell kinetic (S^MM); 1: hybrid S^HMM
                          with the criteria of Sec. 2.2 */
  double thr_g;        /* threshold on the interface norm ||g||_2 */
  double thr_R;        /* threshold on the macroscopic remainder R */
  int32_t r_scale;     /* 0: compare |R| with thr_R (as printed);
                          1: compare eps^2 |R| (the O(eps^2) term of eq.
                          HigherOrderModel) */
  int32_t flux_rule;   /* 0: one flux per interface (mass-conservative);
                          1: the cell-based rule printed in S^HMM */
  double dt;           /* fine step limit; 0 = automatic (stability rule) */
  double cfl_theta;    /* safety factor of the automatic rule (0 -> 0.9) */
  int32_t coarse_kind; /* G: 0 = linearly implicit S^0, 1 = explicit S^0 */
  int32_t coarse_steps;/* G steps per slice (>= 1); the explicit kind uses
                          max(coarse_steps, the steps its stability needs) */
  int32_t lift_order;  /* lifting order L of Def. 1: 1, 2 or 3 (the
                          Chapman-Enskog terms h1..hL of Sec. 2.1 at the
                          interfaces, x-derivatives by Table 1, then the
                          (I - Pi) projection; see mm_lift) */
  int32_t precision;   /* mm_precision */
  int32_t fine_kernel; /* F implementation: 0 = automatic; 1 = streaming
                          (one CTA per state, g in device memory, every
                          option); 2 = resident (g held in the shared memory
                          of a thread-block cluster for the whole call; FP32
                          g, adapt == 0, flux_rule == 0, nv = 8 * {2..32},
                          nx / cluster size a multiple of 32 and <= 256,
                          and a multiple of 4 * 256 / (nv / 8);
                          MM_ERR_INVALID otherwise).  Automatic picks the
                          resident kernel whenever it applies. */
  int32_t fine_vpt;    /* velocity nodes per lane of the streaming kernel:
                          0 = the most that fits (8 in FP32, 4 in FP64, or
                          fewer when nv requires; FP64 offers 8 only
                          where 4 would need more than 32 lanes, nv =
                          256); 1, 2, 4 or 8 forces that lane layout
                          (MM_ERR_INVALID if nv does not allow it).  The
                          batch engine always uses the default. */
} mm_params;

typedef struct mm_ctx mm_ctx;

typedef struct {
  double dt_limit;       /* step limit (rule or params.dt) */
  double dt;             /* step used for the queried span */
  int64_t n_steps;       /* fine steps for the queried span */
  double m2;             /* second velocity moment of the discrete M */
  double a, b;           /* exp(-dt/eps^2), eps (1 - a) */
  size_t state_bytes;    /* bytes of one (rho, g) slice state */
  int32_t vpt;           /* velocity nodes per lane in the fine kernel */
  int32_t lanes;         /* lanes per interface column in the fine kernel */
  int32_t fine_kernel;   /* F implementation mm_fine_propagate runs:
                            1 = streaming, 2 = resident */
  int32_t cluster;       /* CTAs per state (thread-block cluster size) */
} mm_info;

typedef struct {
  int64_t steps;             /* fine steps per state */
  int64_t kinetic_updates;   /* (kinetic interface, v_j) updates, summed over
                                states and steps */
  int64_t full_updates;      /* nx * nv * steps * batch */
  int32_t device_status;     /* mm_status reported by the kernels */
  double elapsed_ms;         /* device time of the call (events) */
  int32_t launches;          /* kernel launches of the call: a batch of more
                                states than the GPU holds at once runs the
                                resident kernel in rounds of step chunks */
} mm_fine_stats;

/* Fill *p with defaults: x_len 1, v_max 8, eps 1, rho_bar NaN, adapt 0,
   thr_g 1e-3, thr_R 1e-2, r_scale 0, flux_rule 0, dt 0, cfl_theta 0.9,
   coarse_kind 0, coarse_steps 1, lift_order 1, precision MM_FP64,
   fine_kernel 0. */
MM_API void mm_params_default(mm_params* p);

/* Create a context for one problem shape.  Validates the parameters,
   builds the velocity grid on the device.  alloc may be NULL.
   Errors: MM_ERR_INVALID (bad parameter or unsupported nv), MM_ERR_CUDA,
   MM_ERR_OOM. */
MM_API mm_status mm_create(const mm_params* p, const mm_alloc* alloc, mm_ctx** out);

/* Release the context and its workspace (synchronises the device). */
MM_API void mm_destroy(mm_ctx* ctx);

/* Step size, step count and constants for a span of t_span.
   Errors: MM_ERR_INVALID (t_span <= 0). */
MM_API mm_status mm_query(const mm_ctx* ctx, double t_span, mm_info* out);

/* F over a span (Sec. 2.3, eq. S^HMM; eq. S^MM when adapt == 0):
   n = ceil(t_span / dt_limit) steps of size t_span / n for every state of
   the batch, all states in one launch (the resident kernel: in rounds of
   step chunks when the batch exceeds the clusters the GPU holds at once;
   stats->launches counts them).  Per step and state: the Poisson law of
   S^MM for E (in the FP32 path with one flux per interface, solved at entry
   and then advanced by the discrete Ampere identity it implies under the
   flux-form density update), the flux J of S^0, the criteria of Sec. 2.2
   and the status
   update of Sec. 2.3 (adapt == 1), the g update on kinetic interfaces
   (upwind transport, (I - Pi) projection, field term, exponential
   relaxation), g = 0 on fluid interfaces, and the density update.
   The status at entry is the kinetic rule applied as if every cell were
   kinetic, so F is a function of (rho_in, g_in) alone.
     rho_in  [batch][nx] double          rho_out [batch][nx] double
     g_in    [batch][nx][nv]             g_out   [batch][nx][nv] (may alias
                                                  g_in)
     mask_out [batch][nx] uint8 or NULL (final cell status)
     stats    NULL, or filled after a stream synchronisation
   Errors: MM_ERR_INVALID (batch < 0, NULL array, t_span <= 0),
   MM_ERR_UNSTABLE (params.dt above the stability rule, or a non-finite
   density in the result: reported through stats->device_status and the
   return value when stats is given), MM_ERR_CUDA, MM_ERR_OOM.
   batch == 0 is a no-op. */
MM_API mm_status mm_fine_propagate(mm_ctx* ctx, int32_t batch, double t_span,
                            const double* rho_in, const void* g_in,
                            double* rho_out, void* g_out, uint8_t* mask_out,
                            mm_fine_stats* stats, void* stream);

/* Size in bytes of the fixed device scratch array of
   mm_fine_propagate_noalloc (64 MiB).  The array is reserved on a device by
   the first mm_create on that device and held until the process exits. */
#define MM_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* mm_fine_propagate for callers that cannot allocate device memory when
   they run F.  The paper has no counterpart: this is a deployment variant of
   the same propagator.  Such callers -- an application whose memory is all
   handed to its own pool, a real-time loop that must not reach the
   allocator or risk an out-of-memory failure mid-run -- create the context
   once at start-up and then call this entry point, which allocates nothing:
   the scratch of the fine kernel (the status word; for the streaming kernel
   also its second step buffer of g, the column arrays when they do not fit
   shared memory, and a copy of g_in when it aliases g_out with an odd step
   count) lives in a static device array of MM_NOALLOC_SCRATCH_BYTES inside
   the library.  mm_create does the set-up with the context's device
   current: it looks up the array's device address (cudaGetSymbolAddress),
   which reserves the array on that device, and loads the kernels of the
   context's launch choice, so no call of this entry point loads anything.
   The call runs the same kernel and launch shape as mm_fine_propagate would
   for the context (the resident kernel where it applies, or the choice of
   mm_autotune), so results are identical.  Arguments are those of
   mm_fine_propagate, with three differences: every array must be a 16-byte
   aligned device pointer (host arrays would need staging buffers);
   stats->elapsed_ms is 0; the call's scratch must fit the array.  Every call
   shares the one array and the array keeps the last call's contents: calls
   that may run at the same time on the GPU (on streams with no ordering
   between them) race on it and must not be issued.
   Errors: MM_ERR_INVALID (as mm_fine_propagate; host or unaligned array;
   scratch needed above MM_NOALLOC_SCRATCH_BYTES, with the size in the
   message), MM_ERR_UNSTABLE, MM_ERR_CUDA. */
MM_API mm_status mm_fine_propagate_noalloc(mm_ctx* ctx, int32_t batch, double t_span,
                                    const double* rho_in, const void* g_in,
                                    double* rho_out, void* g_out, uint8_t* mask_out,
                                    mm_fine_stats* stats, void* stream);

/* Result of mm_autotune: the launch shape chosen and every candidate's
   time (the first 16). */
typedef struct {
  int32_t n_candidates;
  int32_t fine_kernel;       /* chosen: 1 = streaming, 2 = resident */
  int32_t cluster;           /* chosen CTAs per state (resident), else 1 */
  int32_t vpt, lanes;        /* chosen lane layout (streaming kernel) */
  double best_ms;            /* device time of the chosen shape */
  int32_t cand_kernel[16], cand_cluster[16], cand_vpt[16];
  double cand_ms[16];
  double res_entry_steps;    /* resident kernel chosen: measured cost of a
                                step chunk's entry and exit, in steps */
} mm_tune_result;

/* Autotuner of F's launch shape (the numerical scheme, eq. S^HMM of
   Sec. 2.3, is unchanged; only the kernel and its decomposition differ, so
   results agree to rounding).  Times, on the caller's batch, `steps` steps
   of every shape that suits the context -- the resident kernel with each
   cluster size 1, 2, 4, 8 its rules allow, the streaming kernel with each
   lane layout (8, 4, 2 or 1 velocity nodes per lane in FP32; 4, 2, 1 in
   FP64, or 8 where 4 needs more than 32 lanes) -- restricted by
   params.fine_kernel when that is not 0, and keeps the fastest for every
   later mm_fine_propagate and parareal_run of this
   context (mm_query reports it).  When the resident kernel wins, the
   tuner also times one full wave of it for `steps` and for 2 `steps`
   steps; the difference gives the cost of a step chunk's entry and exit
   in steps, which then sets how many steps each launch runs when a batch
   is larger than the GPU holds at once (rounds of step chunks: more
   chunks fill the rounds better, each adds one entry and exit).  The
   batch engine's work-list kernel is not affected.
     rho_in, g_in   inputs as for mm_fine_propagate (not modified)
     rho_out, g_out scratch outputs (must not alias the inputs); they hold
                    the last candidate's result on return
     out            NULL or the choice and the candidates' times
   batch == 0 restores the default choice.  Synchronises the stream.
   Errors: MM_ERR_INVALID (steps < 1, NULL or aliased arrays, no shape),
   MM_ERR_UNSTABLE, MM_ERR_CUDA, MM_ERR_OOM; on error the previous choice
   stays. */
MM_API mm_status mm_autotune(mm_ctx* ctx, int32_t batch, int32_t steps, const double* rho_in,
                             const void* g_in, double* rho_out, void* g_out, mm_tune_result* out,
                             void* stream);

/* Sets the cost of a resident-kernel step chunk's entry and exit, in steps,
   that the launch planner uses when a batch is larger than the GPU holds at
   once (the quantity mm_autotune measures; a later mm_autotune overwrites
   it).  For reproducing a launch plan under a tool that slows every launch
   (a profiler), where the measurement would be inflated.  The results do
   not depend on it: only the number of launches and their step counts.
     entry_steps  >= 0, at most 1000; 0 selects the built-in estimate
   Errors: MM_ERR_INVALID. */
MM_API mm_status mm_set_chunk_entry(mm_ctx* ctx, double entry_steps);

/* G over a span (Sec. 2.3, eq. S^0): coarse_steps linearly implicit steps
   (E frozen from the old density, cyclic tridiagonal solve) or explicit S^0
   steps, for every density of the batch.  rho_in and rho_out may alias.
   Errors: MM_ERR_INVALID, MM_ERR_CUDA, MM_ERR_OOM. */
MM_API mm_status mm_coarse(mm_ctx* ctx, int32_t batch, double t_span,
                    const double* rho_in, double* rho_out, void* stream);

/* Lifting of order L = params.lift_order (Def. 1, Sec. 3.2-3.3): the
   Chapman-Enskog perturbations of the identification in Sec. 2.1 truncated
   at order L, evaluated at the interfaces (interface density averaged as in
   Sec. 3.3), then projected with (I - Pi) so that <g> = 0:
     g = (I - Pi)[eps h1 + eps^2 h2 + eps^3 h3]   (terms up to order L)
     h1 = -v M J,  h2 = (v^2 - 1) M K,
     h3 = v M [dJ/dt - (v^2 - 1) dK/dx - E (3 - v^2) K],
   K = dJ/dx - E J, dJ/dt = d2J/dx2 - rho (J - mean J) - E dJ/dx; E from
   the Poisson law, J the S^0 flux, x-derivatives by the Table 1 stencils
   on the interface grid.  Computed in double; g_out has the context's
   precision.  parareal_run and the batch engine relift with the same order.
   Errors: MM_ERR_INVALID, MM_ERR_CUDA, MM_ERR_OOM. */
MM_API mm_status mm_lift(mm_ctx* ctx, int32_t batch, const double* rho, void* g_out,
                  void* stream);

typedef enum {
  MM_PARAREAL_RHO_LIFT = 0,   /* Algorithm 1: the density is the parareal
                                 unknown; every fine propagation starts from
                                 the lifted density (Sec. 3.2-3.3) */
  MM_PARAREAL_FULL_STATE = 1  /* the fine scheme's state U = (rho, g) is the
                                 unknown: F(U) from the slice's own (rho, g),
                                 G(U) = (G rho, L G rho), the correction on
                                 both parts; converges to the plain
                                 sequential F (parareal_run only) */
} mm_parareal_mode;

typedef struct {
  double t_end;        /* T */
  int32_t n_slices;    /* N_g >= 1 */
  int32_t max_iter;    /* K >= 0 (capped at N_g) */
  double tol;          /* stop when the successive error is below tol */
  int32_t mode;        /* mm_parareal_mode (0 = MM_PARAREAL_RHO_LIFT) */
} mm_parareal_cfg;

typedef struct {
  int32_t iterations;        /* parareal iterations performed */
  double err[64];            /* successive errors (first 64 iterations) */
  double mass_drift;         /* max_n |m^n - m^0| / |m^0| of the result */
  int64_t fine_steps;        /* fine steps per slice */
  int64_t kinetic_updates;   /* summed over all fine propagations */
  double elapsed_ms;         /* device time of the whole call (events) */
  double fine_ms;            /* device time of the fine-propagator launches */
  int32_t fine_launches;     /* fine-propagator kernel launches */
  int32_t kernel_launches;   /* every kernel launch of the call (fine, coarse
                                guess, lifting, correction, mass sums); 0 from
                                mm_batch_take, whose launches serve many solves
                                at once (mm_batch_counters) */
} mm_parareal_stats;

/* Algorithm 1 (Sec. 3.3) with F = S^HMM, G = S^0 and the lifting of order
   params.lift_order: coarse guess, then per iteration k the fine
   propagations of all slices n >= k in one batched launch, the sequential
   correction rho^{n+1,k+1} = F(rho^{n,k}) + (G(rho^{n,k+1}) - G(rho^{n,k}))
   on the device, relifting, and the successive error
   max |rho^{n,k+1} - rho^{n,k}|.  The first slice starts from (rho0, g0);
   later slices from their lifted density.  With cfg.mode ==
   MM_PARAREAL_FULL_STATE the slices carry (rho, g): F starts from the
   slice's own g, and g^{n+1,k+1} = F_g(U^{n,k}) + (L G rho^{n,k+1} -
   L G rho^{n,k}) (the slices' g stay on the device, 2 (N+1) nx nv values).
   rho_slices_out [n_slices + 1][nx] double receives rho^{n,K}.  The call
   synchronises the stream once per iteration (error test and the fine
   launches' status), after the correction: nothing waits between the fine
   launches and the correction.  In density mode,
   when the resident fine kernel runs a batch in rounds of step chunks, part
   of the coarse guess, the lifting and the correction runs on a second
   stream that the context owns, ordered by events against the caller's
   stream; the results are those of the sequential order, and the call
   returns only after that work is complete.
   Errors: MM_ERR_INVALID, MM_ERR_UNSTABLE, MM_ERR_CUDA, MM_ERR_OOM. */
MM_API mm_status parareal_run(mm_ctx* ctx, const mm_parareal_cfg* cfg,
                       const double* rho0, const void* g0,
                       double* rho_slices_out, mm_parareal_stats* stats,
                       void* stream);

/* Algorithm 1's sequential parts as separate calls (Sec. 3.3), for a driver
   that spreads the fine propagations of an iteration over several devices:
   each device runs F (mm_lift, mm_fine_propagate) on its block of the
   slices n = k..N-1, the F results are gathered on every device, and every
   device then runs the same correction, so all of them hold the same
   iterate.  The arithmetic is parareal_run's (same kernels); the per-slice
   fine propagations do not depend on how the slices are split.  Arrays are
   device pointers; rho_bar NaN takes the mean of slice 0 (a host read).

   mm_coarse_guess: the coarse guess rho^{n+1,0} = G(rho^{n,0}),
   n = 0..N-1, with G = S^0 over t_span (mm_coarse's propagator).
     rho_slices [N+1][nx] double: slice 0 given, slices 1..N written
     g_prev     [N+1][nx] double: G(rho^{n,0}) written at index n+1
   Errors: MM_ERR_INVALID (sizes, NULL or host arrays), MM_ERR_CUDA,
   MM_ERR_OOM. */
MM_API mm_status mm_coarse_guess(mm_ctx* ctx, int32_t n_slices, double t_span, double* rho_slices,
                                 double* g_prev, void* stream);

/* mm_parareal_correct: the sequential correction of iteration k,
   rho^{n+1,k+1} = G(rho^{n,k+1}) + F(rho^{n,k}) - G(rho^{n,k}) for
   n = k..N-1 in order, g_prev[n+1] <- G(rho^{n,k+1}), and the successive
   error max_{n,i} |rho^{n,k+1} - rho^{n,k}| into err[0] (device double).
     rho_slices [N+1][nx] in/out; f_rho [N+1][nx], F(rho^{n,k}) at index
     n+1 for n = k..N-1; g_prev [N+1][nx] in/out.
   Errors: MM_ERR_INVALID (k outside [0, N), NULL or host arrays),
   MM_ERR_CUDA, MM_ERR_OOM. */
MM_API mm_status mm_parareal_correct(mm_ctx* ctx, int32_t n_slices, int32_t k, double t_span,
                                     double* rho_slices, const double* f_rho, double* g_prev, double* err,
                                     void* stream);

/* --------------------------------------------------------- many solves --- */

/* A batch of independent parareal solves (Algorithm 1, Sec. 3.3) of any
   shapes, advanced together: each mm_batch_step runs one parareal iteration
   of every unfinished solve in a few launches whatever the number of
   solves -- the coarse guess of newly added solves, every fine propagation
   F the iteration needs, of all solves and slices, as one work list walked
   by a persistent kernel (longest items first; each item lifts its slice
   density in place, so no per-slice perturbation is stored), and the
   sequential corrections with their successive errors.  The coarse guess
   and the corrections run on one CTA per solve, and over a thread-block
   cluster of 8 CTAs for a solve of nx >= 4096 (a power of two up to 32768;
   one launch per grid size): its chain of implicit coarse steps is then
   several times shorter.  Solves may be added
   between steps; a finished solve stays until taken.  The F of a batch is
   the streaming kernel (FP32 g with 8 velocity nodes per lane, or FP64 with
   4: nv / 16, resp. nv / 8, a whole number of lanes, at most 32 lanes).
   Results equal parareal_run's to rounding (the lifting inside the fine
   kernel sums the field in another order) and do not depend on the other
   solves of the batch.  Not thread-safe. */
typedef struct mm_batch mm_batch;

/* Device bytes a solve holds while in a batch (the slice densities, the
   fine results, the previous coarse values and slice 0's perturbation). */
MM_API size_t mm_batch_footprint(const mm_params* p, const mm_parareal_cfg* cfg);
MM_API mm_status mm_batch_create(const mm_alloc* alloc, mm_batch** out);
/* Copy a solve's initial data (host or device arrays rho0 [nx], g0 [nx][nv]
   in the params' precision) into the batch.  The batch runs the density
   mode of Algorithm 1 (cfg.mode must be MM_PARAREAL_RHO_LIFT).
   Errors: MM_ERR_INVALID (parameters, configuration, unsupported nv),
   MM_ERR_OOM, MM_ERR_CUDA. */
MM_API mm_status mm_batch_add(mm_batch* b, const mm_params* p, const mm_parareal_cfg* cfg,
                       const double* rho0, const void* g0, uint64_t* id);
/* One parareal iteration of every unfinished solve; *active (nullable)
   receives the number of solves that were unfinished before the step.
   Synchronises the stream.  Errors: MM_ERR_UNSTABLE (non-finite density),
   MM_ERR_CUDA, MM_ERR_OOM. */
MM_API mm_status mm_batch_step(mm_batch* b, int32_t* active, void* stream);
MM_API mm_status mm_batch_query(mm_batch* b, uint64_t id, int32_t* done);
/* Copy a finished solve's slice densities [n_slices + 1][nx] (host or
   device; NULL to discard) and statistics, and release it.
   Errors: MM_ERR_NOT_READY, MM_ERR_UNKNOWN_TICKET. */
MM_API mm_status mm_batch_take(mm_batch* b, uint64_t id, double* rho_slices_out,
                        mm_parareal_stats* stats);
MM_API size_t mm_batch_bytes(const mm_batch* b);
/* Totals over the batch's life: kinetic cell-updates of all fine
   propagations, fine launches, and their device time (events). */
MM_API mm_status mm_batch_counters(const mm_batch* b, int64_t* kinetic_updates, int32_t* fine_launches,
                            double* fine_ms);
MM_API void mm_batch_destroy(mm_batch* b);

/* parareal_run for n solves at once through a batch: rho0[q], g0[q],
   rho_slices_out[q] are solve q's arrays (host or device); stats may be
   NULL or an array of n.  Errors: as mm_batch_add / mm_batch_step. */
MM_API mm_status parareal_run_many(int32_t n, const mm_params* params, const mm_parareal_cfg* cfgs,
                            const double* const* rho0, const void* const* g0,
                            double* const* rho_slices_out, mm_parareal_stats* stats,
                            void* stream);

/* ------------------------------------------------------------ serving --- */

typedef struct mm_server mm_server;

typedef struct {
  size_t hbm_budget_bytes;   /* admission budget for resident solves */
  int32_t max_slots;         /* solves resident at once */
  int32_t wait_limit_ms;     /* bound on any internal wait */
} mm_server_cfg;

typedef struct {
  mm_params params;
  mm_parareal_cfg cfg;
  const double* rho0;        /* host [nx], copied at submit */
  const void* g0;            /* host [nx][nv] (params.precision), copied */
} mm_request;

typedef struct {
  mm_status status;
  double* rho_T;             /* caller-owned host [nx]: density at t_end */
  int32_t iterations;
  int64_t latency_ns;        /* submit -> result ready */
  int64_t kinetic_updates;
} mm_result;

/* Serving loop with continuous batching.  Two lanes, each one scheduler
   thread that owns an mm_batch and a stream, run rounds: a lane admits its
   queued requests (first come, first served) while their device footprint
   fits hbm_budget_bytes (shared by both lanes) and fewer than max_slots
   solves are resident, runs one parareal iteration of every resident solve
   of the lane (all their fine propagations in one persistent work-list
   launch), and completes the solves that finished.  A request whose
   parareal iteration costs more than 2e10 fine cell-updates (estimated from
   the step rule: nx nv n_slices steps-per-slice) goes to the long lane, the
   others to the short lane; the long lane's launches leave one eighth of
   the SMs to the short lane, so small requests do not wait behind rounds of
   large ones (the short lane uses every SM while no long solve is
   resident).  The lanes' batches keep the cluster layout of the coarse guess
   and corrections for nx >= 16384: a cluster needs 8 free SMs of one GPC,
   which the other lane's launches may hold.  A request's footprint is
   mm_batch_footprint plus its share of
   the fine kernel's step buffers (two states per SM) plus 1 MiB.  Requests
   that arrive while others run join their lane at its next round; a result
   does not depend on the requests it ran with.  If a round fails, the
   solves resident in that lane fail with its status and the lane continues
   with its queue.
   Errors: MM_ERR_INVALID, MM_ERR_CUDA, MM_ERR_OOM. */
MM_API mm_status mm_server_create(const mm_server_cfg* cfg, const mm_alloc* alloc,
                           mm_server** out);
/* Copy the request and queue it.  Errors: MM_ERR_INVALID (bad request, or
   a footprint above the whole budget). */
MM_API mm_status serve_submit(mm_server* s, const mm_request* req, uint64_t* ticket);
/* Wait up to timeout_ms (at most the server's wait_limit_ms) for a result;
   on MM_OK the result (its own status, the density at t_end, iterations,
   latency from submit to completion) is copied into *res and the ticket is
   retired.  Errors: MM_ERR_NOT_READY, MM_ERR_UNKNOWN_TICKET. */
MM_API mm_status serve_poll(mm_server* s, uint64_t ticket, mm_result* res,
                     int32_t timeout_ms);
/* Stop the scheduler, fail queued requests, free device state. */
MM_API mm_status mm_server_destroy(mm_server* s);

/* Measurement helper, not part of the method: the FP32 FMA rate of the
   current device in TFLOP/s (an FMA counts two flops), from independent FMA
   chains on every SM timed with events on `stream` (about 4 ms; synchronises
   the stream).  It is the measured denominator of the resident fine
   kernel's roofline, which is bound by FP32 issue rather than by HBM.
   Errors: MM_ERR_INVALID (NULL), MM_ERR_CUDA. */
MM_API mm_status mm_probe_fp32(double* tflops, void* stream);

/* Message of the last failure on this thread ("" if none). */
MM_API const char* mm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
