/*
 * pic.h -- C ABI of the B300 (sm_103a) implementation of the fully implicit,
 * energy-conserving, unstaggered Lorenz-gauge potential PIC step with the
 * generalized-momentum Higuera-Cary push (arxiv 2609.36383, Part II).
 *
 * One context owns one simulation on one GPU: particles (SoA), mesh
 * potentials and every work buffer live in device memory allocated by the
 * library.  Caller buffers stay caller-owned; get/set copy.  Pointers tagged
 * `on_device` are CUDA device pointers when that flag is 1 and host pointers
 * when it is 0.  A context is not thread-safe; all its work is queued on the
 * stream given in pic_options.cuda_stream (0 = the legacy default stream).
 *
 * Array conventions (all float64 unless stated):
 *   mesh scalars  : Ng = n[0]*n[1]*n[2] values, x fastest (g = i + n0*(j + n1*k));
 *   mesh vectors  : 3*Ng values, component-major (A[c*Ng + g]);
 *   particle x    : dim*N values, dimension-major (x[l*N + i]), absolute positions;
 *   particle u, P : 3*N values, component-major.
 * Ignorable (inactive) dimensions have n = 1 and no derivative (their Fourier
 * symbol is zero); vector fields and momenta always have 3 components.
 *
 * Return codes: 0 on success, else one of the negative PIC_E* codes below; a
 * human-readable message is kept by pic_last_error().
 */
#ifndef PIC_H
#define PIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_EARG (-1)    /* invalid argument or unsupported size */
#define PIC_ENOMEM (-2)  /* device allocation failed */
#define PIC_ECUDA (-3)   /* a CUDA runtime call failed */
#define PIC_EINNER (-4)  /* an inner particle solve failed: iteration limit,
                            non-finite or superluminal velocity (Sec. 4.5) */
#define PIC_EOUTER (-5)  /* outer solve failed: iteration limit or no accepted
                            direction (Algorithm 1) */
#define PIC_ESTATE (-6)  /* call out of order (e.g. pic_step before pic_start) */
#define PIC_ETOOBIG (-7) /* input larger than a fixed-size buffer allows
                            (pic_kinetic_energy_noalloc) */

#define PIC_FP64 0       /* every step of the particle map in FP64 */
#define PIC_MIXED 1      /* push, gather, deposit in FP32; field solve, residual
                            norms and energy sums in FP64 */

typedef struct pic_ctx pic_ctx;

/* Periodic mesh (Sec. 2.3): dim active dimensions, n[l] nodes (a power of
   two, 4..4096) on [x0[l], x0[l] + L[l]); node g sits at x0 + g*L/n. */
typedef struct {
  int dim;
  int n[3];
  double L[3];
  double x0[3];
} pic_grid;

/* Species charge and mass per unit weight: a particle of weight w carries
   q = w*q_s and m = w*m_s (Sec. 5 uses q/m = -1, m = |q|). */
typedef struct {
  double q, m;
} pic_species;

/* Solver and model options.  pic_default_options() fills the paper's values
   (Sec. 5: kappa = sigma1 = sigma2 = 1, 8 inner/outer limits 64/80,
   Anderson M = 4 from iteration 2, beta = 0.5, lambda = 1e-12, backtracking
   alpha = 1 .. 1/64, sufficient decrease 1e-4, growth limit 1.2). */
typedef struct {
  double kappa, sigma1, sigma2; /* Eq. potential-wave; sigma1 = kappa^2 sigma2 */
  double rho_bg;                /* immobile uniform background charge density */
  int project_nyquist;          /* 1: apply the projector of Eq. nyquist-projector */
  int gl_points;                /* Gauss-Legendre points per knot-split orbit piece;
                                   0 = minimal exact count dim+1 */
  int inner_max, outer_max;
  int anderson_m;               /* Anderson history columns M */
  int anderson_start;           /* m_A: outer iterations are counted from 1, and the first
                                   that may take an Anderson direction is iteration m_A
                                   (earlier ones, and any without history, take damped
                                   Picard); pic_report.outer_iters counts the iterations
                                   begun, the last being the one whose tests passed */
  int backtrack_levels;
  double beta, lambda, decrease_coef, growth_limit;
  double tol_abs_ratio;         /* tau_abs = tol * tol_abs_ratio (tau_rel = tol) */
  double inner_tol_scale;       /* inner tolerance = outer tolerance * this */
  int precision;                /* PIC_FP64 or PIC_MIXED */
  double mixed_tol_floor;       /* PIC_MIXED: tolerances are max(tol, this) */
  int sort_every;               /* counting-sort particles by cell every N steps (0 = never) */
  void *cuda_stream;            /* cudaStream_t to queue work on; NULL = a stream the
                                   context creates (blocking, so it orders itself
                                   with the legacy default stream) */
  int inner_warm_start;         /* 0 (default): every map evaluation starts the inner
                                   Picard iteration from v(p^n); 1: later evaluations
                                   of a step start from the previous evaluation's
                                   orbit velocity (fewer inner iterations; H(j) then
                                   depends on the history at the inner tolerance, so
                                   use it with inner_tol_scale < 1) */
  int order;                    /* B-spline degree r of the particle shape: 2 (default,
                                   the paper's production runs, C^1) or 1 (the linear
                                   shapes of the Sec. 5.3 comparison, knots on the nodes) */
  int refine_max;               /* convergence-triggered particle refinement (Sec. 5.3):
                                   a particle whose inner solve fails is retried with
                                   2, 4, .. 2^refine_max equal substeps of the (fixed)
                                   field step, each substep seeing the time-linear
                                   potential of Eq. A-g-s and depositing its orbit
                                   current weighted by its share of the step; 0..3,
                                   default 0 (off) */
  int deterministic_deposit;    /* 1: the orbit current is summed without atomics, node by
                                   node, over nearby particles in an order fixed by their
                                   cell and position (results identical from run to run,
                                   and equal across mesh lines that hold equal particle
                                   configurations); pic_start's point deposits of rho
                                   and J likewise.  Several times the deposit's cost, a
                                   checking mode.  FP64 contexts without refinement and
                                   with at least 8 nodes per active dimension only
                                   (pic_init returns PIC_EARG otherwise), and not in a
                                   batch (pic_batch_init rejects it); default 0 */
  int growth_scaled;            /* Anderson history clearing (Sec. 4.5): the history is
                                   cleared when the RMS residual of an accepted iterate
                                   exceeds growth_limit times the previous one; 0
                                   (default) compares plain RMS residuals, 1 the scaled
                                   RMS residuals of Eq. mixed-nonlinear-tests */
  int host_control;             /* 0 (default): Algorithm 1's decisions are taken on the
                                   device, and a step's whole outer iteration runs as two
                                   CUDA graph launches with one synchronisation at the
                                   end; 1: the host takes them, synchronising after every
                                   map evaluation (the same decisions, for checks).  In a
                                   batch, 1 likewise has the host launch each round and
                                   read the loop state after it */
  int nonlinear_solver;         /* PIC_SOLVER_ANDERSON (default): Algorithm 1's type-II
                                   Anderson iteration; PIC_SOLVER_NEWTON_KRYLOV: inexact
                                   Newton on H(j) - j = 0, each direction from
                                   (I - H'(j)) d = r by GMRES(20) on Jacobian-vector
                                   products (dual-number map evaluations, as
                                   pic_eval_map_jvp), forcing terms of Eisenstat and
                                   Walker (choice 2, gamma 0.9) bounded below by half the
                                   reduction the outer tests still need, the same
                                   backtracking, tests and verifying evaluation as
                                   Algorithm 1.  FP64 contexts with quadratic shapes, no
                                   refinement, the cold inner start and the atomic deposit
                                   (pic_init returns PIC_EARG otherwise); the host drives
                                   the iteration */
  int fp32_first;               /* 1: each step's outer iteration first runs with the
                                   particle map in FP32 arithmetic (the particle state
                                   stays FP64), to max(tol, mixed_tol_floor) and without
                                   verification, then continues in FP64 from that current
                                   to tol, verifies and commits as an FP64 step: FP64
                                   results (energy conserved to the FP64 tolerance) from
                                   fewer FP64 map evaluations.  FP64 contexts with
                                   quadratic shapes, no refinement, the Anderson solver,
                                   device control and the atomic deposit (pic_init
                                   returns PIC_EARG otherwise); default 0 */
} pic_options;

#define PIC_SOLVER_ANDERSON 0
#define PIC_SOLVER_NEWTON_KRYLOV 1

/* Per-step report (Sec. 4.4 diagnostics and solver counters). */
typedef struct {
  double W, K, E_tot;           /* field (Eq. field-energy-section2), kinetic, total energy */
  double rel_dE;                /* (E_tot - E_tot at pic_start) / E_tot at pic_start */
  double gauss_rms, lorenz_rms; /* Eq. constraint-residuals at the new time level */
  double work_residual;         /* Eq. work-diagnostic */
  double chain_rms;             /* Eq. RA-diagnostic */
  double res_scaled_rms, res_scaled_max; /* Eq. mixed-nonlinear-tests at acceptance */
  int outer_iters, map_evals, inner_max;
  double inner_mean;            /* inner iterations of the final map evaluation */
  int status;                   /* return code of the step */
  int refined;                  /* particles of the final map evaluation that needed
                                   substeps (refine_max > 0) */
  int jvp_evals;                /* Jacobian-vector products (dual-number map
                                   evaluations) of the Newton-Krylov solver; 0 otherwise */
  int fp32_evals;               /* map evaluations of the FP32 stage (option fp32_first),
                                   included in map_evals; its iterations are included
                                   in outer_iters */
} pic_report;

/* Fill *opt with the paper's defaults (see pic_options). */
void pic_default_options(pic_options *opt);

/* Create a context: validates the mesh (power-of-two n, dim 1..3), the
   species (1..4, m > 0) and dt > 0, and allocates the mesh buffers on the
   current CUDA device.  opt may be NULL for the defaults.  On failure *out
   is NULL and the return code says why. */
int pic_init(pic_ctx **out, const pic_grid *grid, const pic_species *species,
             int nspecies, double dt, const pic_options *opt);

/* Load N particles (replaces any previous set).  species: N int32 indices
   (NULL = all species 0); x: dim*N absolute positions (wrapped into the box);
   u_or_P: 3*N proper velocities u = gamma v (is_canonical = 0; the canonical
   momentum P = m u + q A_h(x) is formed by pic_start from the projected A,
   Sec. 4.5) or canonical momenta P (is_canonical = 1); w: N weights.
   The context must be started again (pic_start) unless the field state is
   also restored with pic_set_state.  Every species index must lie in
   [0, nspecies): host arrays are checked before anything is copied, device
   arrays by the loading kernel; either way an index out of range returns
   PIC_EARG and leaves the context empty and unstarted. */
int pic_set_particles(pic_ctx *ctx, int64_t n, const int32_t *species,
                      const double *x, const double *u_or_P, int is_canonical,
                      const double *w, int on_device);

/* pic_set_particles with positions in the form the library stores them
   (Sec. 2.4: the nearest node plus the offset from it): cell holds dim*N
   node indices (row l: 0 <= cell < n[l]) and offset dim*N offsets in node
   units, -1/2 <= offset < 1/2; the position along l is
   x0[l] + (cell + offset) * L[l] / n[l].  Particles that should see
   identical arithmetic in different cells (quiet starts, symmetry tests)
   get bit-identical offsets this way, which absolute coordinates far from
   the origin cannot give.  An index or offset out of range returns
   PIC_EARG (host arrays are checked before anything is copied, device
   arrays by the loading kernel) and leaves the context empty and
   unstarted.  Everything else is as for pic_set_particles. */
int pic_set_particles_local(pic_ctx *ctx, int64_t n, const int32_t *species,
                            const int32_t *cell, const double *offset, const double *u_or_P,
                            int is_canonical, const double *w, int on_device);

/* Initial vector potential A and its time derivative U (3*Ng each; NULL =
   zero).  Both are projected by pic_start. */
int pic_set_potentials(pic_ctx *ctx, const double *A, const double *U, int on_device);

/* Prepare step 0 (Sec. 4.5 and the initial constraints of Sec. 2.3): project
   A and U, form P from u if needed, deposit rho^0 and J^0 with point shapes
   and project them, solve phi^0 from Gauss's law and psi^0 from the Lorenz
   gauge, and record the initial total energy.  *out (may be NULL) receives
   the diagnostics at step 0. */
int pic_start(pic_ctx *ctx, pic_report *out);

/* One implicit GM-HC-CN step, Algorithm 1, with tau_rel = tol and
   tau_abs = tol*tol_abs_ratio.  On PIC_EINNER / PIC_EOUTER the accepted state
   is unchanged and *out still carries the counters. */
int pic_step(pic_ctx *ctx, double tol, pic_report *out);

/* One evaluation of the outer map H(j) = P J_orb(j) (Sec. 4.5) from the
   accepted state, without committing anything.  j, H: 3*Ng; vbar, Pnew:
   3*N converged orbit velocities and candidate canonical momenta, in the
   order the particles were loaded; inner_counts: N int32 (-1 = failed).
   Any output pointer may be NULL. */
int pic_eval_map(pic_ctx *ctx, const double *j, double tol, double *H,
                 double *vbar, double *Pnew, int32_t *inner_counts, int on_device);

/* One evaluation of the outer map and its directional derivative (a
   Jacobian-vector product): H = H(j) as pic_eval_map computes it, and
   dH = H'(j) dj.  The field step's tangent is its CN update of dj with zero
   accepted state; the particle part is differentiated in forward mode
   through the inner Picard fixed point, the knot-split orbit integrals, the
   GM-HC push and the deposit.  For a Newton-Krylov outer solver in place of
   the Picard/Anderson iteration of Algorithm 1 (the paper has no tangent).
   j, dj, H, dH: 3*Ng; H or dH may be NULL.  Only FP64 contexts with
   quadratic shapes, no refinement and the cold inner start (PIC_EARG
   otherwise).  Allocates its scratch (about (dim + 15) * 16 bytes per
   particle) for the call and frees it. */
int pic_eval_map_jvp(pic_ctx *ctx, const double *j, const double *dj, double tol,
                     double *H, double *dH, int on_device);

/* The adjoint of one map evaluation (a vector-Jacobian product): H = H(j)
   as pic_eval_map computes it and jbar = H'(j)^T ybar.  Transposed from the
   output back: the Nyquist projector (symmetric); the orbit deposit, whose
   transpose is the orbit gather of the cotangent current; each particle's
   inner fixed point vbar = Phi(vbar, F) by implicit differentiation (a
   3 x 3 solve with (I - Phi_vbar)^T); the gather, whose transpose scatters
   the push's transpose-vector product with the gather's orbit weights; and
   the CN field step, mode by mode.  The paper differentiates nothing; the
   dot product <ybar, H'(j) dj> of pic_eval_map_jvp equals <jbar, dj>.
   j, ybar, H, jbar: 3*Ng; H or jbar may be NULL.  FP64 contexts with
   quadratic shapes, no refinement and the cold inner start only (PIC_EARG
   otherwise).  Allocates its scratch (about 15 * 8 bytes per particle and
   12 * 8 + 12 * 16 bytes per mesh node) for the call and frees it. */
int pic_eval_map_vjp(pic_ctx *ctx, const double *j, const double *ybar, double tol,
                     double *H, double *jbar, int on_device);

/* The adjoint of one implicit step (reverse mode): given the cotangents of
   the state after the step, Sbar' = (xbar', Pbar', fbar'), the cotangents of
   the state before it, Sbar = (dS'/dS)^T Sbar'.  The state is what
   pic_get_particles and pic_get_potentials return: absolute positions x
   (dim*N, load order), canonical momenta P (3*N, load order), and the
   real-space potentials packed as fbar = [phi (Ng), psi (Ng), A (3*Ng),
   U (3*Ng), rho (Ng)] (9*Ng).  The step's fixed point j* = H(j*, S) is
   differentiated implicitly: Sbar = G_S^T Sbar' + H_S^T lambda with
   (I - H_j^T) lambda = G_j^T Sbar', where G commits the particles and the
   field step; lambda by restarted GMRES(20) to relative residual
   max(tol, 1e-12) (*gmres_iters receives the operator applications; may be
   NULL).  The call recomputes the step from the current state (pic_step at
   tol, orbits recomputed in the backward pass) and leaves the state
   unchanged; a forward sensitivity (pic_tangent_begin) is dropped.  Input
   cotangents may be NULL (zero); outputs may be NULL (not wanted).  Chain
   calls over a run's saved checkpoint images (pic_checkpoint_save), last
   step first, for the gradient of a function of the final state with
   respect to the initial one.  FP64, quadratic shapes, no refinement, cold
   inner start only (PIC_EARG otherwise); PIC_EINNER / PIC_EOUTER if the
   step or the adjoint solve fails.  The paper differentiates nothing. */
int pic_step_vjp(pic_ctx *ctx, double tol, const double *xbar1, const double *Pbar1,
                 const double *fbar1, double *xbar0, double *Pbar0, double *fbar0,
                 int *gmres_iters, int on_device);

/* Autotuner of the counting-sort interval (sort_every): from the current
   accepted state, each of the ncand candidate intervals (>= 0; 0 = never
   sort) runs `steps` implicit steps at tolerance tol, timed with CUDA events
   on the context's stream, each starting from the same snapshot of the
   state (the checkpoint image's content, held in device memory), with the
   particles sorted by cell first when the candidate sorts; then the
   snapshot is restored, so
   the state is exactly the one before the call (same bits, particle order
   and step count), sort_every is set to the fastest candidate and returned
   in *best.  ms_per_step (ncand entries, may be NULL) receives each
   candidate's time.  The statistics of pic_get_stats exclude the tuning
   steps.  A forward sensitivity (pic_tangent_begin) is dropped.
   The paper has no autotuner; the interval trades the sort's cost against
   the gathers' locality.  A failing step returns its code with the state
   restored and sort_every unchanged. */
int pic_tune_sort(pic_ctx *ctx, double tol, int steps, const int *candidates, int ncand,
                  int *best, double *ms_per_step);

/* Forward sensitivity of the whole step (the tangent of the state with
   respect to one parameter of the initial condition), for gradients of
   quantities after many steps.  pic_tangent_begin seeds it at the started
   state: du, the tangent of the particles' mechanical u (3*N, load order),
   and dA, dU, the tangents of the initial potentials (3*Ng each); any may
   be NULL (zero).  The positions carry no seed.  The seed follows pic_start:
   dA and dU are projected, dP = m du + q (P dA)_h(x), dphi from Gauss's law,
   dpsi from the Lorenz gauge, drho = 0.  From then on every successful
   pic_step also advances the tangent: the tangent dj of the converged
   current solves (I - H_j) dj = H_s dS (implicit differentiation of the
   fixed point j = H(j; S) of Sec. 4.5 with respect to the accepted state S)
   by restarted GMRES(20) on JVPs until |dj - H_j dj - H_S dS| is at most
   max(tol, 1e-12) times the larger of |dj| and |H_S dS| (or stalls below
   1e-9 of it: the attainable accuracy where the net tangent current is a
   small part of its gross terms);
   the tangents of vbar, P^{n+1} and the CN field step follow from dj.  A
   tangent solve that does not converge fails the step with PIC_EOUTER and
   leaves state and tangent unchanged.  FP64 contexts with quadratic shapes,
   no refinement and the cold inner start only (PIC_EARG otherwise).
   Allocates about (dim + 3) * 8 + (dim + 15) * 16 bytes per particle and
   about 1.4 kB per mesh node; pic_tangent_end (or pic_start,
   pic_set_particles, pic_set_state, pic_free) releases it. */
int pic_tangent_begin(pic_ctx *ctx, const double *du, const double *dA, const double *dU,
                      int on_device);
int pic_tangent_end(pic_ctx *ctx);

/* The tangent of the accepted state: dx (dim*N, physical units) and dP
   (3*N) in load order, dA, dU (3*Ng, real space), and the tangents of the
   kinetic, field and total energy (dK, dW; their sum is conserved exactly
   as E_tot is).  Any pointer may be NULL.  PIC_ESTATE without a tangent.
   gmres_iters (may be NULL) receives the Krylov iterations of the last
   step's tangent solve. */
int pic_get_tangent(pic_ctx *ctx, double *dx, double *dP, double *dA, double *dU, double *dK,
                    double *dW, int *gmres_iters, int on_device);

int64_t pic_num_particles(const pic_ctx *ctx);

/* Copy the accepted particle state out, in load order.  Any pointer may be NULL. */
int pic_get_particles(pic_ctx *ctx, double *x, double *P, double *w,
                      int32_t *species, int on_device);

/* Proper velocities u = p / m (so v = u / gamma) of the accepted particles,
   with the mechanical momentum p = P - q A_h(x) (Eq. rel-P-def), in load
   order: 3*N values, component-major. */
int pic_get_velocities(pic_ctx *ctx, double *u, int on_device);

/* Copy the accepted mesh state out: phi, psi, rho (Ng), A, U (3*Ng) at the
   current time level and J (3*Ng), the accepted current J^{n-1/2} that seeds
   the next outer iteration.  Any pointer may be NULL. */
int pic_get_potentials(pic_ctx *ctx, double *phi, double *psi, double *A,
                       double *U, double *rho, double *J, int on_device);

/* Restore a full accepted state (checkpoint/resume): particles as canonical
   momenta in load order and the mesh state as returned by pic_get_particles
   and pic_get_potentials.  E0 is the reference total energy for rel_dE.
   No projection or constraint solve is applied. */
int pic_set_state(pic_ctx *ctx, int64_t n, const int32_t *species, const double *x,
                  const double *P, const double *w, const double *phi,
                  const double *psi, const double *A, const double *U,
                  const double *rho, const double *J, double E0, int on_device);

/* Checkpoint image: the accepted state of a context as bytes, for exact
   resume (library support; the paper has no counterpart).  Unlike
   pic_set_state, which takes the real-space arrays of pic_get_* and passes
   them through an FFT, the image holds the device state itself (particles in
   storage order as cell index + in-cell offset, potentials as spectral
   coefficients), so a context that loads it continues with the very bits the
   saving context had.  With deterministic_deposit = 1 the resumed steps equal
   the uninterrupted run's bit for bit; with the atomic deposit they agree to
   the deposit's summation-order rounding.

   Layout, all little-endian: this 256-byte header, then 13 sections, each
   starting on a 16-byte boundary (zero padding counted in the checksum):
     cell  int32  [dim][np]    nearest node per active dimension
     off   real   [dim][np]    offset in node units, in [-1/2, 1/2]
     P     real   [3][np]      canonical momentum
     w     f64    [np]         weight
     sp    int32  [np]         species
     id    int64  [np]         load-order index (a permutation of 0..np-1)
     phi, psi, rho  c128 [Ng] each; A, U  c128 [3][Ng]  unnormalised DFT
                               coefficients of the accepted potentials
     A     f64    [3][Ng]      A^n in real space
     J     f64    [3][Ng]      accepted current (seed of the next outer solve)
   where real is f64 for PIC_FP64 and f32 for PIC_MIXED and c128 is a
   (re, im) pair of f64. */
typedef struct {
  char magic[8];          /* "PICCKPT1" */
  uint32_t version;       /* 1 */
  uint32_t header_bytes;  /* 256 */
  uint64_t total_bytes;   /* header + payload */
  uint64_t checksum;      /* 64-bit FNV-1a of the bytes after the header */
  int32_t dim, n[3];      /* mesh; n = 1 in ignorable dimensions */
  int32_t precision;      /* PIC_FP64 or PIC_MIXED */
  int32_t nspecies;
  int32_t sort_every;     /* sort interval in effect (pic_tune_sort may set it) */
  int32_t reserved0;
  double L[3], x0[3];
  double q[4], m[4];      /* species charge and mass per unit weight */
  double dt;              /* time step of the saving context (not checked on load) */
  double E0;              /* reference total energy for rel_dE */
  int64_t np;             /* particles */
  int64_t steps_done;     /* accepted steps since pic_start (sort schedule) */
  uint8_t reserved[48];
} pic_checkpoint_header;

/* Size in bytes of the image of the context's current state. */
int pic_checkpoint_bytes(const pic_ctx *ctx, uint64_t *bytes);

/* Write the image into a HOST buffer of exactly pic_checkpoint_bytes bytes
   (PIC_EARG otherwise; PIC_ESTATE before pic_start).  Synchronises the
   context's stream. */
int pic_checkpoint_save(pic_ctx *ctx, void *image, uint64_t bytes);

/* Validate an image on the host (no context and no GPU needed): magic,
   version, sizes, checksum, and every value later used as an index (cells
   inside the mesh, offsets within [-1/2, 1/2], species below nspecies, the
   load-order indices a permutation).  Fills *header (may be NULL) and, on
   PIC_EARG, writes the reason into why (may be NULL, why_len bytes with the
   terminating zero). */
int pic_checkpoint_inspect(const void *image, uint64_t bytes, pic_checkpoint_header *header,
                           char *why, int why_len);

/* Replace the context's state with a validated image.  The context must have
   the image's mesh (dim, n, L, x0 bitwise), precision and species (q, m);
   its options (tolerances, deposit mode, ...) stay its own except the sort
   interval, which the image sets.  Any forward sensitivity is dropped.
   PIC_EARG (nothing changed) for an invalid or foreign image; after a
   PIC_ECUDA / PIC_ENOMEM the context refuses pic_step (PIC_ESTATE) until a
   state is set again. */
int pic_checkpoint_load(pic_ctx *ctx, const void *image, uint64_t bytes);

/* The knot-jump regularity diagnostic of Sec. 5.3 on the accepted fields.
   The field interpolants F_h = sum_g F_g S_r(x - x_g) use the context's
   particle shape (degree r = pic_options.order).  They are probed at every
   knot of S_r (the nodes for r = 1, the cell midpoints for r = 2) along
   every active axis, at +-eps node units along the axis (the paper uses
   eps = 1e-8).  The other coordinates sit half a cell from their own knots:
   on the node for r = 2, at the cell centre for r = 1.  *E_jump receives
   the largest |E(+) - E(-)| of E_shape = -grad phi_h - U_h (Euclidean
   norm), *G_jump the largest |G(+) - G(-)| of G = grad A_h (Frobenius
   norm, columns per active dimension).  O(1) jumps mark the discontinuous
   first derivatives of r = 1, O(eps) the continuous ones of r = 2.
   PIC_EARG unless 0 < eps < 1/4; PIC_ESTATE before pic_start. */
int pic_knot_jumps(pic_ctx *ctx, double eps, double *E_jump, double *G_jump);

/* Counters of the work this context has done (library profiling support;
   the paper has no counterpart).  map_ms is the device time of the particle
   map kernel (inner solves + deposit) measured with CUDA events recorded on
   the context's stream around each launch. */
typedef struct {
  int64_t launches;      /* kernels launched by this context */
  int64_t map_launches;  /* particle-map kernel launches */
  double map_ms;         /* summed device time of those launches, ms */
  int64_t pushes;        /* particles x map evaluations */
  int64_t inner_iters;   /* summed inner Picard iterations */
  int64_t pieces;        /* summed knot-split orbit pieces walked (gathers and deposits) */
  int64_t refined;       /* particle solves that needed substeps (refine_max > 0) */
} pic_stats;

int pic_get_stats(const pic_ctx *ctx, pic_stats *out);
int pic_reset_stats(pic_ctx *ctx);

/* Measured fused-multiply-add throughput of the current device in FLOP/s
   (2 per FMA), for PIC_FP64 or PIC_MIXED (FP32): many independent FMA chains
   in every thread of a grid of 8 CTAs per SM, timed with CUDA events.  Used
   as the ALU roofline of the particle map, which no library reports.
   Allocates one small device buffer and frees it before returning. */
int pic_fma_throughput(int precision, double *flops_per_s);

/* Kinetic energy sum_i m_i kappa^2 (gamma_i - 1), with p_i = P_i - q_i A_h(x_i),
   of a particle set in a mesh vector potential, computed WITHOUT ALLOCATING
   ANY MEMORY.  The paper has no counterpart: this entry point serves callers
   that cannot call cudaMalloc, for example code whose memory pool or arena
   owns the whole device, code inside a latency-critical loop where an
   allocation would synchronize the device, or frameworks that forbid
   allocations on their hot path.  It computes the same sum that pic_start
   and pic_step report as K, but needs no context.
   Arguments: grid, species (1..4) and kappa as for pic_init; n particles
   with DEVICE arrays sp (n int32 indices in [0, nspecies), NULL = species
   0; an index out of range returns PIC_EARG, and is never used to index
   the species tables), x (dim*n absolute
   positions), P (3*n canonical momenta), w (n weights), A (3*Ng vector
   potential, layout as in pic_get_potentials); *K_out is a HOST double.
   The interpolation A_h uses the quadratic shape (order 2, the default).
   All work is queued on cuda_stream (NULL = legacy default stream) and the
   call returns after that stream has finished it.
   Scratch: a fixed array of 16,386 doubles (128 KiB) of device memory
   inside the library, which every GPU that loads the library holds until
   the process exits; at most PIC_NOALLOC_MAX_PARTICLES particles, larger n
   returns PIC_ETOOBIG.  The first call on each device looks up that array's
   device address (cudaGetSymbolAddress) with the device current and keeps
   it for the process; make that first call before any stream capture.  A
   reset of the device's primary context (cudaDeviceReset) reloads the
   library's device code at a new address, so after one the cached address
   is stale: do not call this function again in a process that has reset
   the device.  Every call shares the array, so calls whose
   work overlaps on the GPU (other streams, other threads) race and must be
   serialised by the caller.  Returns PIC_EARG on invalid arguments and
   PIC_ECUDA if a launch or copy fails. */
#define PIC_NOALLOC_MAX_PARTICLES (16384LL * 256LL)
int pic_kinetic_energy_noalloc(const pic_grid *grid, const pic_species *species, int nspecies,
                               double kappa, int64_t n, const int32_t *sp, const double *x,
                               const double *P, const double *w, const double *A,
                               double *K_out, void *cuda_stream);

const char *pic_last_error(const pic_ctx *ctx);
void pic_free(pic_ctx *ctx);

/* ---- batched ensembles of 1D3V problems -----------------------------------
 *
 * A pic_batch advances B independent one-dimensional (1D3V) problems with
 * one implicit step each per call: the step of pic_step (Algorithm 1 with the
 * GM-HC push, orbit deposit and CN field solve of Sec. 2-4) applied to every
 * instance, with every phase of the step run as one GPU launch over all
 * instances and the outer solver's decisions (accept, backtrack, Anderson or
 * damped Picard, verify) taken on the device per instance.  The paper has no
 * ensemble driver; each instance computes exactly what a single-problem
 * context with the same grid, particles, species, dt and options computes
 * (up to the summation order of its reductions).
 *
 * Instances share the species, dt and options and differ in their mesh
 * (n[b] nodes, a power of two 4..1024, on [x0[b], x0[b] + L[b])) and
 * particles (np[b], 0 allowed).  Every array below is in HOST memory, and
 * the layouts are those of the single-problem calls with dim = 1.  The batch
 * owns all device memory; options.cuda_stream selects the stream (NULL = a
 * stream the batch creates).  options.anderson_m may be at most 8.
 * Not thread-safe. */
typedef struct pic_batch pic_batch;

/* Create a batch of B instances (1 <= B <= 65536).  x0 may be NULL (all 0);
   opt may be NULL for the defaults.  Returns PIC_EARG for invalid sizes or
   options, PIC_ENOMEM if the device allocations fail. */
int pic_batch_init(pic_batch **out, int B, const int *n, const double *L, const double *x0,
                   const int64_t *np, const pic_species *species, int nspecies, double dt,
                   const pic_options *opt);

/* Stage the initial data of instance inst (0 <= inst < B): np[inst]
   particles as for pic_set_particles with is_canonical = 0 (species may be
   NULL; x: np absolute positions; u: 3*np proper velocities; w: np weights)
   and the potentials A, U (3*n[inst] each, NULL = zero) as for
   pic_set_potentials.  The data are copied; pic_batch_start consumes them. */
int pic_batch_set_instance(pic_batch *b, int inst, const int32_t *species, const double *x,
                           const double *u, const double *w, const double *A, const double *U);

/* pic_start for every instance (projection, P from u, rho^0 and J^0, the
   initial constraints, the reference energy).  Every instance must have been
   staged (else PIC_ESTATE).  reports: B entries or NULL. */
int pic_batch_start(pic_batch *b, pic_report *reports);

/* One implicit step of every instance with tau_rel = tol, tau_abs =
   tol*tol_abs_ratio.  Instances whose step fails keep their accepted state
   (as pic_step does) and report PIC_EINNER / PIC_EOUTER in their
   pic_report.status; the others commit.  Returns PIC_OK when every instance
   succeeded, else the status of the first failed instance.
   reports: B entries or NULL. */
int pic_batch_step(pic_batch *b, double tol, pic_report *reports);

int64_t pic_batch_num_particles(const pic_batch *b, int inst);

/* The accepted particles of one instance in load order (x: np; P: 3*np
   canonical momenta; w: np; species: np int32).  Any pointer may be NULL. */
int pic_batch_get_particles(pic_batch *b, int inst, double *x, double *P, double *w,
                            int32_t *species);

/* The accepted mesh state of one instance as in pic_get_potentials
   (phi, psi, rho: n; A, U, J: 3*n).  Any pointer may be NULL. */
int pic_batch_get_potentials(pic_batch *b, int inst, double *phi, double *psi, double *A,
                             double *U, double *rho, double *J);

/* Work counters as pic_get_stats (map_ms is not measured: 0). */
int pic_batch_get_stats(const pic_batch *b, pic_stats *out);
int pic_batch_reset_stats(pic_batch *b);

const char *pic_batch_last_error(const pic_batch *b);
void pic_batch_free(pic_batch *b);

#ifdef __cplusplus
}
#endif
#endif
