/*
 * pic_oracle.h -- interface of the plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This header, pic_oracle.c and the Python loader
 * beside them exist to check the CUDA path; only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load them.  The oracle
 * shares no source with the CUDA library and must never be used as a
 * fallback for it.
 *
 * The oracle follows the paper (arxiv 2609.36383, "An Energy-Conserving
 * Unstaggered Electromagnetic-Potential PIC Method, Part II") literally:
 *   - CN potential update and continuity        (Sec. 2.3, Eqs. CN-field, cn-continuity)
 *   - orbit-averaged shape, deposit, gather    (Sec. 2.4, Eqs. orbit-average-shape .. orbit-gather-general)
 *   - orbit discrete gradient D_i A            (Sec. 2.5, Eq. D-def)
 *   - HC magnetic map                          (Sec. 3.2, Defs. hc-normalized, hc-dimensional)
 *   - GM-HC canonical step                     (Sec. 3.4, Eq. gmhc-step)
 *   - secant velocity and orbit velocity       (Sec. 4.1-4.2, Eqs. Vdg, vbar-energy)
 *   - diagnostics                              (Sec. 4.4)
 *   - Nyquist projector, outer Anderson / inner Picard solve (Sec. 4.5, Algorithm 1)
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_SPECIES 4
#define ORC_MAX_ANDERSON 8

typedef struct {
  int dim;            /* active spatial dimensions, 1..3 */
  int n[3];           /* nodes per dimension (1 for ignorable dims) */
  double L[3];        /* periodic lengths */
  double x0[3];       /* position of node 0 */
  double dt, kappa, sigma1, sigma2;
  double rho_bg;      /* uniform immobile background charge density */
  int project;        /* 1: Nyquist projection on (Sec. 4.5) */
  int gl_points;      /* Gauss-Legendre points per knot-split piece (paper: 8) */
  int inner_max, outer_max;
  int anderson_m, anderson_start, backtrack_levels;
  double beta, lambda, decrease_coef, growth_limit, tol_abs_ratio, inner_tol_scale;
  int nspecies;
  double q[ORC_MAX_SPECIES], m[ORC_MAX_SPECIES]; /* per unit weight */
  int order;          /* B-spline degree r of the particle shape: 2 (paper's
                         production runs) or 1 (Sec. 5.3 comparison) */
  int refine_max;     /* convergence-triggered particle refinement (Sec. 5.3):
                         a particle whose solve fails is retried with 2, 4, ..
                         2^refine_max equal substeps; 0 = off */
  int growth_scaled;  /* Anderson history clearing (Sec. 4.5, reading R8): 0
                         compares plain RMS residuals of successive iterates,
                         1 the scaled RMS of Eq. mixed-nonlinear-tests */
} orc_params;

/* Per-iteration record of the outer solve (test support): entry k describes
   outer iteration k (0-based).  j: the iterate at which its tests ran
   (cap * 3Ng doubles, may be NULL); srms, smax: its scaled residuals;
   kind: the accepted direction (0 damped Picard, 1 Anderson, 2 damped
   Picard after a rejected Anderson direction; -1 none: the tests passed or
   the step failed); alpha: the accepted step length; mh: history columns
   after the update.  n receives the number of entries written. */
typedef struct {
  int cap;
  double *j;
  double *srms, *smax;
  int *kind;
  double *alpha;
  int *mh;
  int n;
} orc_outer_trace;

typedef struct {
  double W, K, E_tot, rel_dE;
  double gauss_rms, lorenz_rms, work_residual, chain_rms;
  double res_scaled_rms, res_scaled_max;
  int outer_iters, map_evals, inner_max;
  double inner_mean;
  int status;
} orc_report;

/* status codes (shared meaning with the product ABI, separate definitions) */
#define ORC_OK 0
#define ORC_EARG (-1)
#define ORC_EINNER (-4)
#define ORC_EOUTER (-5)

void *orc_create(const orc_params *prm);
void orc_free(void *h);
int orc_set_particles(void *h, long np, const int *species, const double *x,
                      const double *u_or_P, int canonical, const double *w);
int orc_set_potentials(void *h, const double *A, const double *U);
int orc_start(void *h, orc_report *rep);
int orc_step(void *h, double tol, orc_report *rep);
int orc_eval_map(void *h, const double *j, double tol, double *H, double *vbar,
                 double *Pnew, int *inner_counts);
long orc_num_particles(void *h);
/* particles that needed substeps (refinement) in the last map evaluation */
long orc_last_refined(void *h);
int orc_get_particles(void *h, double *x, double *P, double *w, int *species);
int orc_get_fields(void *h, double *phi, double *psi, double *A, double *U,
                   double *rho, double *J);
int orc_set_fields(void *h, const double *phi, const double *psi, const double *A,
                   const double *U, const double *rho, const double *J);

/* The knot-jump regularity diagnostic of Sec. 5.3: the maxima, over every
   knot of the field interpolant (the particle shape's knots) along every
   active axis, with the other coordinates half a cell from their knots
   (on nodes for S_2, at cell centres for S_1), of the two-sided
   differences at +-eps node units of E_shape = -grad phi_h - U_h
   (Euclidean norm) and of grad A_h (Frobenius norm). */
int orc_knot_jumps(void *h, double eps, double *E_jump, double *G_jump);

/* A full accepted state, as after pic_start or a step (test support, no
   arithmetic): particles with canonical momenta and every mesh array; the
   context is then started, so orc_step continues from it. */
int orc_set_state(void *h, long np, const int *species, const double *x, const double *P,
                  const double *w, const double *phi, const double *psi, const double *A,
                  const double *U, const double *rho, const double *J);

/* The tests of Eq. mixed-nonlinear-tests on Ng nodes of 3 components
   (component-major): scaled RMS and scaled maximum-node residual. */
void orc_scaled_tests(long Ng, const double *r, const double *H, const double *j,
                      double tau_r, double tau_a, double *srms, double *smax);

/* The outer solve of Algorithm 1 (the same code orc_step runs) on the affine
   stand-in map H(j) = M j + b, M row-major 3Ng x 3Ng: j holds the initial
   trial current and returns the last iterate; tau_rel = tol, tau_abs =
   tol * tol_abs_ratio; only the outer-solver fields of prm are read.  tr
   (may be NULL) records each iteration. */
int orc_outer_affine(const orc_params *prm, long Ng, const double *M, const double *b,
                     double *j, double tol, orc_outer_trace *tr, orc_report *rep);

/* unit-level pieces, exposed so that tests can pin them one by one */
double orc_S2(double xi);
double orc_dS2(double xi);
double orc_S1(double xi);
double orc_dS1(double xi);
void orc_gauss_legendre(int n, double *nodes, double *weights);
void orc_dft(int dim, const int *n, const double *in_re, const double *in_im,
             double *out_re, double *out_im, int inverse);
void orc_hc_map(const double *um, const double *B, double qdt_2m, double *up,
                double *gamma_hc);
void orc_push(const double *Pn, const double *Am, const double *Ap,
              const double *gphi, const double *D, const double *vbar, double q,
              double m, double kappa, double dt, double *pminus, double *pplus,
              double *Pnp1, double *vnew);
int orc_orbit_data(void *h, const double *x, const double *vbar,
                   const double *gradphi, const double *An, const double *Anp1,
                   const double *Uhalf, double *gphi, double *Ubar, double *D,
                   double *Aplus, double *Aminus, double *Sbar_sum);
int orc_field_solve(void *h, const double *j, double *gradphi_half,
                    double *A_np1, double *U_half, double *phi_np1,
                    double *psi_np1, double *U_np1, double *rho_np1);
double orc_field_energy(void *h, const double *phi, const double *A,
                        const double *U);
void orc_constraint_rms(void *h, const double *phi, const double *psi,
                        const double *A, const double *U, const double *rho,
                        double *gauss_rms, double *lorenz_rms);
void orc_project(void *h, double *f, int ncomp);
int orc_deposit(void *h, const double *vbar, double *Jorb);
int orc_eval_particles(void *h, const double *j, double tol, long nidx, const long *idx,
                       double *vbar, double *Pnew, int *inner_counts);

#ifdef __cplusplus
}
#endif
#endif
