/*
 * pic_oracle.c -- plain, slow, FP64 CPU oracle of the GM-HC-CN implicit PIC step.
 *
 * TEST INFRASTRUCTURE ONLY (see pic_oracle.h).  Every routine below restates a
 * definition of the paper (arxiv 2609.36383) in the most direct form available:
 *   - Fourier transforms are direct O(N^2) DFTs along each axis;
 *   - the quadratic B-spline is evaluated from its (.)_+ formula on every node
 *     of a window that covers the whole orbit;
 *   - orbit integrals use 8-point Gauss-Legendre on every knot-split piece;
 *   - the CN potential update is a 2x2 linear solve per Fourier mode (Cramer);
 *   - the outer/inner nonlinear solve follows Algorithm 1.
 * Nothing here is blocked, fused or reordered for speed.  OpenMP only splits
 * the particle loop.
 *
 * Readings of points the paper leaves open (also listed in the design notes):
 *   R1 knots of S_2 are the half-integer node coordinates;
 *   R3 the first-derivative symbol is 0 on an even-grid Nyquist index;
 *   R5 every map evaluation starts its inner iteration from v(p^n), so that
 *      H(j) is a function of j alone (this matches the 3-5 inner iterations
 *      the paper reports for the final evaluation of each step);
 *   R6 inner test: max_c |vnew_c - v_c| <= tau_abs + tau_rel max_c |vnew_c|;
 *   R7 the deposit uses the final orbit velocity and its own orbit weights;
 *   R8 Anderson: iterations are counted from 1, and iteration m_A
 *      (anderson_start) is the first that may take an Anderson direction;
 *      before it, and whenever no history exists, damped Picard (j + beta r);
 *      history cleared when the regularised Gram solve is not finite or the
 *      unscaled RMS residual grows by more than growth_limit;
 *   R9 tau_rel = tol, tau_abs = tol * tol_abs_ratio;
 *   R10 phi^0 and psi^0 come from the Gauss and Lorenz constraints;
 *   R11 the first trial current is the projected point deposit of q v S(x);
 *   R12 particle charge and mass are weight times the species values;
 *   R15 degree-one shapes (Sec. 5.3 comparison) have their knots on the nodes;
 *   R16 convergence-triggered refinement (Sec. 5.3): a particle whose solve
 *       fails is retried with 2, 4, .. equal substeps of the field step; a
 *       substep over [s_a, s_b] of the step sees A(s) = (1 - s) A^n + s A^{n+1}
 *       (the time-linear potential of Eq. A-g-s) and the step's grad phi^{1/2},
 *       starts its Picard iteration from v(p) at its own start, and deposits
 *       its orbit current with weight (s_b - s_a) (orbit-averaged current).
 */
#include "pic_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define WMAX 12   /* widest node window per dimension of one orbit */
#define GLMAX 32
#define REFMAX 3  /* largest refinement level: 2^3 substeps */

typedef struct {
  orc_params p;
  int Ng;
  double dx[3], dV;
  long np;
  int *sp;
  double *x;        /* x[l*np + i], wrapped into [x0, x0+L) */
  double *P;        /* canonical momentum, P[c*np + i] */
  double *w;
  double *u_mech;   /* mechanical input (proper velocity) awaiting orc_start */
  int pending_mech;
  double *phi, *psi, *A, *U, *rho, *J; /* accepted state; A,U,J are 3*Ng */
  /* step work */
  double *vbar, *v0, *Am, *pn, *Pnew;
  int *iters;
  int *nsub;        /* substeps of each particle's accepted solve (R16) */
  long refined;     /* particles that needed substeps in the last evaluation */
  double gl_t[GLMAX], gl_w[GLMAX];
  double E0;
  int started;
} orc;

/* ------------------------------------------------------------------ */
/* quadratic B-spline, Sec. 4.5 (displayed S_2 formula)                */
/* ------------------------------------------------------------------ */
static double pos(double a) { return a > 0.0 ? a : 0.0; }

double orc_S2(double xi) {
  double a = fabs(xi);
  double p1 = pos(1.5 - a), p2 = pos(0.5 - a);
  return 0.5 * (p1 * p1 - 3.0 * p2 * p2);
}

/* derivative of S_2 with respect to xi */
double orc_dS2(double xi) {
  double a = fabs(xi);
  double sg = (xi > 0.0) ? 1.0 : ((xi < 0.0) ? -1.0 : 0.0);
  return sg * (-pos(1.5 - a) + 3.0 * pos(0.5 - a));
}

/* linear B-spline S_1(xi) = (1 - |xi|)_+ (Sec. 5.3, degree r = 1) */
double orc_S1(double xi) { return pos(1.0 - fabs(xi)); }

/* derivative of S_1 with respect to xi (one-sided values at its knots are
   never needed: quadrature points lie inside knot-split pieces) */
double orc_dS1(double xi) {
  if (fabs(xi) >= 1.0) return 0.0;
  return xi > 0.0 ? -1.0 : (xi < 0.0 ? 1.0 : 0.0);
}

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rule on [0,1] by Newton's method on P_n (textbook)   */
/* ------------------------------------------------------------------ */
void orc_gauss_legendre(int n, double *nodes, double *weights) {
  for (int i = 0; i < n; i++) {
    double x = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; k++) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (n == 1) { p1 = x; p0 = 1.0; }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; k++) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (n == 1) { p1 = x; p0 = 1.0; }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
    }
    nodes[i] = 0.5 * (1.0 + x);
    weights[i] = 1.0 / ((1.0 - x * x) * dp * dp); /* (2/((1-x^2)P'^2)) / 2 */
  }
}

/* ------------------------------------------------------------------ */
/* direct DFT along every active axis; forward unnormalised,          */
/* inverse scaled by 1/N per axis (reading R3)                         */
/* ------------------------------------------------------------------ */
void orc_dft(int dim, const int *n, const double *in_re, const double *in_im,
             double *out_re, double *out_im, int inverse) {
  int N0 = n[0], N1 = dim > 1 ? n[1] : 1, N2 = dim > 2 ? n[2] : 1;
  int total = N0 * N1 * N2;
  for (int g = 0; g < total; g++) {
    out_re[g] = in_re[g];
    out_im[g] = in_im ? in_im[g] : 0.0;
  }
  double sgn = inverse ? 1.0 : -1.0;
  for (int a = 0; a < dim; a++) {
    int N = n[a];
    int stride = (a == 0) ? 1 : (a == 1 ? N0 : N0 * N1);
    double *c = (double *)malloc(sizeof(double) * N);
    double *s = (double *)malloc(sizeof(double) * N);
    double *lr = (double *)malloc(sizeof(double) * N);
    double *li = (double *)malloc(sizeof(double) * N);
    for (int m = 0; m < N; m++) {
      c[m] = cos(2.0 * M_PI * m / N);
      s[m] = sin(2.0 * M_PI * m / N);
    }
    for (int g = 0; g < total; g++) {
      if ((g / stride) % N != 0) continue; /* g starts a line along axis a */
      for (int k = 0; k < N; k++) {
        double sr = 0.0, si = 0.0;
        for (int m = 0; m < N; m++) {
          int idx = (int)(((long)k * m) % N);
          double re = out_re[g + m * stride], im = out_im[g + m * stride];
          sr += re * c[idx] - im * sgn * s[idx];
          si += im * c[idx] + re * sgn * s[idx];
        }
        lr[k] = sr;
        li[k] = si;
      }
      for (int k = 0; k < N; k++) {
        out_re[g + k * stride] = inverse ? lr[k] / N : lr[k];
        out_im[g + k * stride] = inverse ? li[k] / N : li[k];
      }
    }
    free(c); free(s); free(lr); free(li);
  }
}

/* ------------------------------------------------------------------ */
/* spectral helpers                                                    */
/* ------------------------------------------------------------------ */
static int mod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

/* integer wave index along an axis, the derivative symbol (R3) and the
   Nyquist flag of Eq. nyquist-projector */
static double ksym(const orc *o, int a, int k, int *nyq) {
  int N = o->p.n[a];
  *nyq = 0;
  if (a >= o->p.dim) return 0.0;
  if (N % 2 == 0 && k == N / 2) { *nyq = 1; return 0.0; }
  int kk = (k < N / 2 || (N % 2 == 1 && k <= N / 2)) ? k : k - N;
  return 2.0 * M_PI * kk / o->p.L[a];
}

static void mode_of(const orc *o, int g, double kt[3], int *is_nyq) {
  int i0 = g % o->p.n[0];
  int i1 = (g / o->p.n[0]) % o->p.n[1];
  int i2 = g / (o->p.n[0] * o->p.n[1]);
  int idx[3] = {i0, i1, i2};
  *is_nyq = 0;
  for (int a = 0; a < 3; a++) {
    int ny = 0;
    kt[a] = ksym(o, a, idx[a], &ny);
    if (ny) *is_nyq = 1;
  }
}

static void fwd(const orc *o, const double *f, double complex *F) {
  double *re = (double *)malloc(sizeof(double) * o->Ng);
  double *im = (double *)malloc(sizeof(double) * o->Ng);
  orc_dft(o->p.dim, o->p.n, f, NULL, re, im, 0);
  for (int g = 0; g < o->Ng; g++) F[g] = re[g] + I * im[g];
  free(re); free(im);
}

static void inv(const orc *o, const double complex *F, double *f) {
  double *re = (double *)malloc(sizeof(double) * o->Ng);
  double *im = (double *)malloc(sizeof(double) * o->Ng);
  double *ore = (double *)malloc(sizeof(double) * o->Ng);
  double *oim = (double *)malloc(sizeof(double) * o->Ng);
  for (int g = 0; g < o->Ng; g++) { re[g] = creal(F[g]); im[g] = cimag(F[g]); }
  orc_dft(o->p.dim, o->p.n, re, im, ore, oim, 1);
  for (int g = 0; g < o->Ng; g++) f[g] = ore[g];
  free(re); free(im); free(ore); free(oim);
}

static double complex *cbuf(const orc *o) {
  return (double complex *)calloc((size_t)o->Ng, sizeof(double complex));
}

/* Nyquist projector, Eq. nyquist-projector, applied per component */
void orc_project(void *h, double *f, int ncomp) {
  orc *o = (orc *)h;
  if (!o->p.project) return;
  double complex *F = cbuf(o);
  for (int c = 0; c < ncomp; c++) {
    fwd(o, f + (size_t)c * o->Ng, F);
    for (int g = 0; g < o->Ng; g++) {
      double kt[3]; int nq;
      mode_of(o, g, kt, &nq);
      if (nq) F[g] = 0.0;
    }
    inv(o, F, f + (size_t)c * o->Ng);
  }
  free(F);
}

/* ------------------------------------------------------------------ */
/* mesh energy and constraint residuals (Eqs. field-energy-section2,  */
/* constraint-residuals), evaluated on the mesh in real space          */
/* ------------------------------------------------------------------ */
static void grad_real(const orc *o, const double *f, double *out3) {
  double complex *F = cbuf(o), *G = cbuf(o);
  fwd(o, f, F);
  for (int a = 0; a < 3; a++) {
    for (int g = 0; g < o->Ng; g++) {
      double kt[3]; int nq;
      mode_of(o, g, kt, &nq);
      G[g] = I * kt[a] * F[g];
    }
    inv(o, G, out3 + (size_t)a * o->Ng);
  }
  free(F); free(G);
}

static void curl_real(const orc *o, const double *A, double *B) {
  double complex *Ah[3], *G = cbuf(o);
  for (int a = 0; a < 3; a++) { Ah[a] = cbuf(o); fwd(o, A + (size_t)a * o->Ng, Ah[a]); }
  for (int a = 0; a < 3; a++) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    for (int g = 0; g < o->Ng; g++) {
      double kt[3]; int nq;
      mode_of(o, g, kt, &nq);
      G[g] = I * (kt[b] * Ah[c][g] - kt[c] * Ah[b][g]);
    }
    inv(o, G, B + (size_t)a * o->Ng);
  }
  for (int a = 0; a < 3; a++) free(Ah[a]);
  free(G);
}

static double div_real_at(const orc *o, const double *V, double *out) {
  double complex *Vh[3], *G = cbuf(o);
  for (int a = 0; a < 3; a++) { Vh[a] = cbuf(o); fwd(o, V + (size_t)a * o->Ng, Vh[a]); }
  for (int g = 0; g < o->Ng; g++) {
    double kt[3]; int nq;
    mode_of(o, g, kt, &nq);
    G[g] = I * (kt[0] * Vh[0][g] + kt[1] * Vh[1][g] + kt[2] * Vh[2][g]);
  }
  inv(o, G, out);
  for (int a = 0; a < 3; a++) free(Vh[a]);
  free(G);
  return 0.0;
}

double orc_field_energy(void *h, const double *phi, const double *A, const double *U) {
  orc *o = (orc *)h;
  size_t N3 = (size_t)3 * o->Ng;
  double *E = (double *)malloc(sizeof(double) * N3);
  double *B = (double *)malloc(sizeof(double) * N3);
  grad_real(o, phi, E);
  for (size_t k = 0; k < N3; k++) E[k] = -E[k] - U[k];
  curl_real(o, A, B);
  double W = 0.0;
  for (int g = 0; g < o->Ng; g++) {
    double e2 = 0.0, b2 = 0.0;
    for (int a = 0; a < 3; a++) {
      e2 += E[(size_t)a * o->Ng + g] * E[(size_t)a * o->Ng + g];
      b2 += B[(size_t)a * o->Ng + g] * B[(size_t)a * o->Ng + g];
    }
    W += (e2 / (2.0 * o->p.sigma1) + b2 / (2.0 * o->p.sigma2)) * o->dV;
  }
  free(E); free(B);
  return W;
}

void orc_constraint_rms(void *h, const double *phi, const double *psi, const double *A,
                        const double *U, const double *rho, double *gauss_rms,
                        double *lorenz_rms) {
  orc *o = (orc *)h;
  size_t N3 = (size_t)3 * o->Ng;
  double *E = (double *)malloc(sizeof(double) * N3);
  double *dE = (double *)malloc(sizeof(double) * o->Ng);
  double *dA = (double *)malloc(sizeof(double) * o->Ng);
  grad_real(o, phi, E);
  for (size_t k = 0; k < N3; k++) E[k] = -E[k] - U[k];
  div_real_at(o, E, dE);
  div_real_at(o, A, dA);
  double sg = 0.0, sl = 0.0;
  for (int g = 0; g < o->Ng; g++) {
    double rg = dE[g] - o->p.sigma1 * rho[g];
    double rl = psi[g] / (o->p.kappa * o->p.kappa) + dA[g];
    sg += rg * rg;
    sl += rl * rl;
  }
  *gauss_rms = sqrt(sg / o->Ng);
  *lorenz_rms = sqrt(sl / o->Ng);
  free(E); free(dE); free(dA);
}

/* ------------------------------------------------------------------ */
/* CN potential update (Eq. CN-field) with continuity                  */
/* (Eq. cn-continuity), mode by mode; each mode's 2x2 system is solved */
/* by Cramer's rule                                                    */
/* ------------------------------------------------------------------ */
static void cn_pair(double dt, double kap2, double k2, double complex fn,
                    double complex gn, double complex src, double complex *f1,
                    double complex *g1) {
  /* unknowns (f1, g1):  f1 - dt/2 g1            = fn + dt/2 gn
                         dt kap2 k2/2 f1 + g1    = gn - dt kap2 k2/2 fn + dt kap2 src */
  double a11 = 1.0, a12 = -0.5 * dt, a21 = 0.5 * dt * kap2 * k2, a22 = 1.0;
  double complex r1 = fn + 0.5 * dt * gn;
  double complex r2 = gn - 0.5 * dt * kap2 * k2 * fn + dt * kap2 * src;
  double det = a11 * a22 - a12 * a21;
  *f1 = (r1 * a22 - a12 * r2) / det;
  *g1 = (a11 * r2 - a21 * r1) / det;
}

int orc_field_solve(void *h, const double *j, double *gradphi_half, double *A_np1,
                    double *U_half, double *phi_np1, double *psi_np1, double *U_np1,
                    double *rho_np1) {
  orc *o = (orc *)h;
  int Ng = o->Ng;
  double dt = o->p.dt, kap2 = o->p.kappa * o->p.kappa;
  double complex *jh[3], *Ah[3], *Uh[3], *rh = cbuf(o), *ph = cbuf(o), *qh = cbuf(o);
  for (int a = 0; a < 3; a++) {
    jh[a] = cbuf(o); Ah[a] = cbuf(o); Uh[a] = cbuf(o);
    fwd(o, j + (size_t)a * Ng, jh[a]);
    fwd(o, o->A + (size_t)a * Ng, Ah[a]);
    fwd(o, o->U + (size_t)a * Ng, Uh[a]);
  }
  fwd(o, o->rho, rh);
  fwd(o, o->phi, ph);
  fwd(o, o->psi, qh);
  double complex *out_g[3], *out_A[3], *out_Uh[3], *out_U1[3];
  double complex *out_phi = cbuf(o), *out_psi = cbuf(o), *out_rho = cbuf(o);
  for (int a = 0; a < 3; a++) {
    out_g[a] = cbuf(o); out_A[a] = cbuf(o); out_Uh[a] = cbuf(o); out_U1[a] = cbuf(o);
  }
  for (int g = 0; g < Ng; g++) {
    double kt[3]; int nq;
    mode_of(o, g, kt, &nq);
    if (nq && o->p.project) continue; /* projected space: every output is zero */
    double k2 = kt[0] * kt[0] + kt[1] * kt[1] + kt[2] * kt[2];
    double complex divj = I * (kt[0] * jh[0][g] + kt[1] * jh[1][g] + kt[2] * jh[2][g]);
    double complex r1 = rh[g] - dt * divj;
    double complex rhalf = 0.5 * (rh[g] + r1);
    double complex f1, g1;
    cn_pair(dt, kap2, k2, ph[g], qh[g], o->p.sigma1 * rhalf, &f1, &g1);
    out_phi[g] = f1;
    out_psi[g] = g1;
    out_rho[g] = r1;
    double complex phalf = 0.5 * (ph[g] + f1);
    for (int a = 0; a < 3; a++) {
      double complex A1, U1;
      cn_pair(dt, kap2, k2, Ah[a][g], Uh[a][g], o->p.sigma2 * jh[a][g], &A1, &U1);
      out_A[a][g] = A1;
      out_U1[a][g] = U1;
      out_Uh[a][g] = 0.5 * (Uh[a][g] + U1);
      out_g[a][g] = I * kt[a] * phalf;
    }
  }
  for (int a = 0; a < 3; a++) {
    if (gradphi_half) inv(o, out_g[a], gradphi_half + (size_t)a * Ng);
    if (A_np1) inv(o, out_A[a], A_np1 + (size_t)a * Ng);
    if (U_half) inv(o, out_Uh[a], U_half + (size_t)a * Ng);
    if (U_np1) inv(o, out_U1[a], U_np1 + (size_t)a * Ng);
  }
  if (phi_np1) inv(o, out_phi, phi_np1);
  if (psi_np1) inv(o, out_psi, psi_np1);
  if (rho_np1) inv(o, out_rho, rho_np1);
  for (int a = 0; a < 3; a++) {
    free(jh[a]); free(Ah[a]); free(Uh[a]);
    free(out_g[a]); free(out_A[a]); free(out_Uh[a]); free(out_U1[a]);
  }
  free(rh); free(ph); free(qh); free(out_phi); free(out_psi); free(out_rho);
  return 0;
}

/* the particle shape of degree o->p.order, its derivative, the half-width
   of its support and the offset of its knots from the nodes (R1, R15) */
static double shp(const orc *o, double xi) { return o->p.order == 1 ? orc_S1(xi) : orc_S2(xi); }
static double dshp(const orc *o, double xi) {
  return o->p.order == 1 ? orc_dS1(xi) : orc_dS2(xi);
}
static double shp_rad(const orc *o) { return o->p.order == 1 ? 1.0 : 1.5; }
static double knot_off(const orc *o) { return o->p.order == 1 ? 0.0 : 0.5; }

/* ------------------------------------------------------------------ */
/* point interpolant A_h(x) = sum_g A_g S_g(x), Eq. mesh-interpolant   */
/* ------------------------------------------------------------------ */
static void node_coord(const orc *o, const double *xp, double *u) {
  for (int l = 0; l < 3; l++)
    u[l] = (l < o->p.dim) ? (xp[l] - o->p.x0[l]) / o->dx[l] : 0.0;
}

static void interp_point(const orc *o, const double *u, const double *F, int ncomp,
                         double *out) {
  int d = o->p.dim, lo[3] = {0, 0, 0}, wn[3] = {1, 1, 1};
  const double rad = shp_rad(o);
  for (int l = 0; l < d; l++) {
    lo[l] = (int)floor(u[l] - rad);
    wn[l] = (int)ceil(u[l] + rad) - lo[l] + 1;
  }
  for (int c = 0; c < ncomp; c++) out[c] = 0.0;
  for (int c2 = 0; c2 < wn[2]; c2++)
    for (int c1 = 0; c1 < wn[1]; c1++)
      for (int c0 = 0; c0 < wn[0]; c0++) {
        int cc[3] = {c0, c1, c2};
        double S = 1.0;
        int gi[3] = {0, 0, 0};
        for (int l = 0; l < d; l++) {
          S *= shp(o, u[l] - (lo[l] + cc[l]));
          gi[l] = mod(lo[l] + cc[l], o->p.n[l]);
        }
        if (S == 0.0) continue;
        size_t g = (size_t)gi[0] + (size_t)o->p.n[0] * (gi[1] + (size_t)o->p.n[1] * gi[2]);
        for (int c = 0; c < ncomp; c++) out[c] += F[(size_t)c * o->Ng + g] * S;
      }
}

/* ------------------------------------------------------------------ */
/* orbit integrals of Sec. 2.4-2.5 for one particle, with knot-split   */
/* Gauss-Legendre quadrature (Sec. 2.5 end; Sec. 5: 8 points/piece)    */
/* ------------------------------------------------------------------ */
typedef struct {
  double gphi[3], Ubar[3], D[9], Aplus[3], Sbar_sum;
  int lo[3], wn[3];
  double Sbar[WMAX * WMAX * WMAX];
} orbit_t;

/* The orbit x(s) = x + s dt_orb vbar, s in [0, 1], over a particle time
   step dt_orb (the field step, or a substep of it, R16); An and Anp1 are the
   potentials at the start and end of that time interval. */
static int orbit_eval(const orc *o, const double *xp, const double *vb, double dt_orb,
                      const double *gradphi, const double *An, const double *Anp1,
                      const double *Uhalf, orbit_t *ob, int want_sbar) {
  int d = o->p.dim, Ng = o->Ng;
  double u0[3], del[3];
  const double rad = shp_rad(o), ko = knot_off(o);
  node_coord(o, xp, u0);
  for (int l = 0; l < 3; l++) {
    del[l] = (l < d) ? dt_orb * vb[l] / o->dx[l] : 0.0;
    ob->lo[l] = 0;
    ob->wn[l] = 1;
  }
  for (int l = 0; l < d; l++) {
    double a = fmin(u0[l], u0[l] + del[l]), b = fmax(u0[l], u0[l] + del[l]);
    ob->lo[l] = (int)floor(a - rad);
    ob->wn[l] = (int)ceil(b + rad) - ob->lo[l] + 1;
    if (ob->wn[l] > WMAX) return -1;
  }
  /* knots crossed by the unwrapped straight orbit, Eq. rel-orbit */
  double bs[4 * WMAX + 2];
  int nb = 0;
  bs[nb++] = 0.0;
  bs[nb++] = 1.0;
  for (int l = 0; l < d; l++) {
    if (del[l] == 0.0) continue;
    double a = fmin(u0[l], u0[l] + del[l]), b = fmax(u0[l], u0[l] + del[l]);
    for (double hk = floor(a - ko) + 1.0 + ko; hk < b; hk += 1.0) {
      if (hk <= a) continue;
      bs[nb++] = (hk - u0[l]) / del[l];
    }
  }
  for (int i = 1; i < nb; i++) /* insertion sort */
    for (int k = i; k > 0 && bs[k - 1] > bs[k]; k--) {
      double t = bs[k]; bs[k] = bs[k - 1]; bs[k - 1] = t;
    }
  memset(ob->gphi, 0, sizeof ob->gphi);
  memset(ob->Ubar, 0, sizeof ob->Ubar);
  memset(ob->D, 0, sizeof ob->D);
  int nw = ob->wn[0] * ob->wn[1] * ob->wn[2];
  if (want_sbar) memset(ob->Sbar, 0, sizeof(double) * nw);
  double sv[3][WMAX], dv[3][WMAX];
  for (int pc = 0; pc + 1 < nb; pc++) {
    double sa = bs[pc], sb = bs[pc + 1];
    if (!(sb > sa)) continue;
    for (int qp = 0; qp < o->p.gl_points; qp++) {
      double s = sa + (sb - sa) * o->gl_t[qp];
      double wt = (sb - sa) * o->gl_w[qp];
      for (int l = 0; l < 3; l++)
        for (int c = 0; c < ob->wn[l]; c++) {
          if (l < d) {
            double xi = u0[l] + s * del[l] - (ob->lo[l] + c);
            sv[l][c] = shp(o, xi);
            dv[l][c] = dshp(o, xi) / o->dx[l];
          } else {
            sv[l][c] = 1.0;
            dv[l][c] = 0.0;
          }
        }
      for (int c2 = 0; c2 < ob->wn[2]; c2++)
        for (int c1 = 0; c1 < ob->wn[1]; c1++)
          for (int c0 = 0; c0 < ob->wn[0]; c0++) {
            int cc[3] = {c0, c1, c2};
            double S = sv[0][c0] * sv[1][c1] * sv[2][c2];
            double dS[3];
            dS[0] = dv[0][c0] * sv[1][c1] * sv[2][c2];
            dS[1] = sv[0][c0] * dv[1][c1] * sv[2][c2];
            dS[2] = sv[0][c0] * sv[1][c1] * dv[2][c2];
            int gi[3];
            for (int l = 0; l < 3; l++) gi[l] = mod(ob->lo[l] + cc[l], o->p.n[l]);
            size_t g = (size_t)gi[0] + (size_t)o->p.n[0] * (gi[1] + (size_t)o->p.n[1] * gi[2]);
            if (want_sbar) ob->Sbar[c0 + ob->wn[0] * (c1 + ob->wn[1] * c2)] += wt * S;
            for (int a = 0; a < 3; a++) {
              if (gradphi) ob->gphi[a] += wt * S * gradphi[(size_t)a * Ng + g];
              if (Uhalf) ob->Ubar[a] += wt * S * Uhalf[(size_t)a * Ng + g];
              double Aas = (1.0 - s) * An[(size_t)a * Ng + g] + s * Anp1[(size_t)a * Ng + g];
              for (int jj = 0; jj < 3; jj++) ob->D[a * 3 + jj] += wt * Aas * dS[jj];
            }
          }
    }
  }
  double u1[3];
  for (int l = 0; l < 3; l++) u1[l] = u0[l] + del[l];
  interp_point(o, u1, Anp1, 3, ob->Aplus);
  ob->Sbar_sum = 0.0;
  if (want_sbar)
    for (int k = 0; k < nw; k++) ob->Sbar_sum += ob->Sbar[k];
  return 0;
}

/* ------------------------------------------------------------------ */
/* HC magnetic map, Definition hc-normalized (Eqs. hc-tau-sigma ..    */
/* hc-explicit)                                                        */
/* ------------------------------------------------------------------ */
static void cross(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

void orc_hc_map(const double *um, const double *B, double qdt_2m, double *up,
                double *gamma_hc) {
  double tau[3] = {qdt_2m * B[0], qdt_2m * B[1], qdt_2m * B[2]};
  double gm = sqrt(1.0 + dot3(um, um));
  double tau2 = dot3(tau, tau);
  double sigma = gm * gm - tau2;
  double ut = dot3(um, tau);
  double g = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (tau2 + ut * ut))));
  double t[3] = {tau[0] / g, tau[1] / g, tau[2] / g};
  double t2 = dot3(t, t);
  double s[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2), 2.0 * t[2] / (1.0 + t2)};
  double uxt[3], ustar[3], uxs[3];
  cross(um, t, uxt);
  for (int c = 0; c < 3; c++) ustar[c] = um[c] + uxt[c];
  cross(ustar, s, uxs);
  for (int c = 0; c < 3; c++) up[c] = um[c] + uxs[c];
  if (gamma_hc) *gamma_hc = g;
}

/* secant velocity, Eq. Vdg */
static void vdg(const double *pa, const double *pb, double m, double kappa, double *v) {
  double mk2 = m * m * kappa * kappa;
  double ga = sqrt(1.0 + dot3(pa, pa) / mk2), gb = sqrt(1.0 + dot3(pb, pb) / mk2);
  for (int c = 0; c < 3; c++) v[c] = (pa[c] + pb[c]) / (m * (ga + gb));
}

/* GM-HC canonical step with frozen orbit data, Eq. gmhc-step, followed
   by the orbit velocity of Eqs. electric-work-velocities, vbar-energy.
   D is row-major: D[l*3+j] = [D_i A]_{l j}. */
void orc_push(const double *Pn, const double *Am, const double *Ap, const double *gphi,
              const double *D, const double *vbar, double q, double m, double kappa,
              double dt, double *pminus, double *pplus, double *Pnp1, double *vnew) {
  double Aep[3], Dv[3];
  for (int c = 0; c < 3; c++) {
    Aep[c] = 0.5 * (Am[c] + Ap[c]);
    Dv[c] = D[c * 3 + 0] * vbar[0] + D[c * 3 + 1] * vbar[1] + D[c * 3 + 2] * vbar[2];
  }
  for (int c = 0; c < 3; c++)
    pminus[c] = Pn[c] - q * Aep[c] - 0.5 * q * dt * gphi[c] + 0.5 * q * dt * Dv[c];
  /* K = D^T - D (Eq. D-split-skew); B_eff = (K23, -K13, K12) (Eq. beff-KA) */
  double K[9];
  for (int l = 0; l < 3; l++)
    for (int jj = 0; jj < 3; jj++) K[l * 3 + jj] = D[jj * 3 + l] - D[l * 3 + jj];
  double Beff[3] = {K[1 * 3 + 2], -K[0 * 3 + 2], K[0 * 3 + 1]};
  double um[3], up[3];
  for (int c = 0; c < 3; c++) um[c] = pminus[c] / (m * kappa);
  orc_hc_map(um, Beff, q * dt / (2.0 * m), up, NULL);
  for (int c = 0; c < 3; c++) pplus[c] = m * kappa * up[c];
  for (int c = 0; c < 3; c++)
    Pnp1[c] = pplus[c] + q * Aep[c] - 0.5 * q * dt * gphi[c] + 0.5 * q * dt * Dv[c];
  double pn[3], pnp1[3], vm[3], vp[3];
  for (int c = 0; c < 3; c++) {
    pn[c] = Pn[c] - q * Am[c];
    pnp1[c] = Pnp1[c] - q * Ap[c];
  }
  vdg(pminus, pn, m, kappa, vm);
  vdg(pnp1, pplus, m, kappa, vp);
  for (int c = 0; c < 3; c++) vnew[c] = 0.5 * (vm[c] + vp[c]);
}

/* ------------------------------------------------------------------ */
/* state management                                                    */
/* ------------------------------------------------------------------ */
void *orc_create(const orc_params *prm) {
  if (!prm || prm->dim < 1 || prm->dim > 3 || prm->nspecies < 1 ||
      prm->nspecies > ORC_MAX_SPECIES || prm->gl_points < 1 || prm->gl_points > GLMAX ||
      (prm->order != 1 && prm->order != 2) || prm->refine_max < 0 || prm->refine_max > REFMAX ||
      prm->anderson_m < 0 || prm->anderson_m > ORC_MAX_ANDERSON)
    return NULL;
  orc *o = (orc *)calloc(1, sizeof(orc));
  o->p = *prm;
  for (int l = prm->dim; l < 3; l++) { o->p.n[l] = 1; o->p.L[l] = 1.0; o->p.x0[l] = 0.0; }
  o->Ng = o->p.n[0] * o->p.n[1] * o->p.n[2];
  o->dV = 1.0;
  for (int l = 0; l < 3; l++) {
    o->dx[l] = o->p.L[l] / o->p.n[l];
    if (l < o->p.dim) o->dV *= o->dx[l];
  }
  size_t N = (size_t)o->Ng;
  o->phi = (double *)calloc(N, sizeof(double));
  o->psi = (double *)calloc(N, sizeof(double));
  o->rho = (double *)calloc(N, sizeof(double));
  o->A = (double *)calloc(3 * N, sizeof(double));
  o->U = (double *)calloc(3 * N, sizeof(double));
  o->J = (double *)calloc(3 * N, sizeof(double));
  orc_gauss_legendre(o->p.gl_points, o->gl_t, o->gl_w);
  return o;
}

static void free_particles(orc *o) {
  free(o->sp); free(o->x); free(o->P); free(o->w); free(o->u_mech);
  free(o->vbar); free(o->v0); free(o->Am); free(o->pn); free(o->Pnew); free(o->iters);
  free(o->nsub);
  o->sp = NULL; o->x = o->P = o->w = o->u_mech = NULL;
  o->vbar = o->v0 = o->Am = o->pn = o->Pnew = NULL; o->iters = NULL;
}

void orc_free(void *h) {
  orc *o = (orc *)h;
  if (!o) return;
  free_particles(o);
  free(o->phi); free(o->psi); free(o->rho); free(o->A); free(o->U); free(o->J);
  free(o);
}

long orc_num_particles(void *h) { return ((orc *)h)->np; }

long orc_last_refined(void *h) { return ((orc *)h)->refined; }

static double wrap_pos(const orc *o, int l, double x) {
  double r = fmod(x - o->p.x0[l], o->p.L[l]);
  if (r < 0) r += o->p.L[l];
  if (r >= o->p.L[l]) r -= o->p.L[l];
  return o->p.x0[l] + r;
}

int orc_set_particles(void *h, long np, const int *species, const double *x,
                      const double *u_or_P, int canonical, const double *w) {
  orc *o = (orc *)h;
  free_particles(o);
  o->np = np;
  size_t n = (size_t)np;
  o->sp = (int *)calloc(n ? n : 1, sizeof(int));
  o->x = (double *)calloc(3 * (n ? n : 1), sizeof(double));
  o->P = (double *)calloc(3 * (n ? n : 1), sizeof(double));
  o->w = (double *)calloc(n ? n : 1, sizeof(double));
  o->u_mech = (double *)calloc(3 * (n ? n : 1), sizeof(double));
  o->vbar = (double *)calloc(3 * (n ? n : 1), sizeof(double));
  o->v0 = (double *)calloc(3 * (n ? n : 1), sizeof(double));
  o->Am = (double *)calloc(3 * (n ? n : 1), sizeof(double));
  o->pn = (double *)calloc(3 * (n ? n : 1), sizeof(double));
  o->Pnew = (double *)calloc(3 * (n ? n : 1), sizeof(double));
  o->iters = (int *)calloc(n ? n : 1, sizeof(int));
  o->nsub = (int *)calloc(n ? n : 1, sizeof(int));
  for (size_t i = 0; i < n; i++) {
    o->sp[i] = species ? species[i] : 0;
    if (o->sp[i] < 0 || o->sp[i] >= o->p.nspecies) return ORC_EARG;
    o->w[i] = w[i];
    for (int l = 0; l < o->p.dim; l++) o->x[l * n + i] = wrap_pos(o, l, x[l * n + i]);
    for (int c = 0; c < 3; c++) {
      if (canonical) o->P[c * n + i] = u_or_P[c * n + i];
      else o->u_mech[c * n + i] = u_or_P[c * n + i];
    }
  }
  o->pending_mech = !canonical;
  o->started = 0;
  return ORC_OK;
}

int orc_set_potentials(void *h, const double *A, const double *U) {
  orc *o = (orc *)h;
  size_t N3 = (size_t)3 * o->Ng;
  for (size_t k = 0; k < N3; k++) {
    o->A[k] = A ? A[k] : 0.0;
    o->U[k] = U ? U[k] : 0.0;
  }
  o->started = 0;
  return ORC_OK;
}

int orc_get_particles(void *h, double *x, double *P, double *w, int *species) {
  orc *o = (orc *)h;
  size_t n = (size_t)o->np;
  if (x) memcpy(x, o->x, sizeof(double) * o->p.dim * n);
  if (P) memcpy(P, o->P, sizeof(double) * 3 * n);
  if (w) memcpy(w, o->w, sizeof(double) * n);
  if (species) memcpy(species, o->sp, sizeof(int) * n);
  return ORC_OK;
}

int orc_get_fields(void *h, double *phi, double *psi, double *A, double *U, double *rho,
                   double *J) {
  orc *o = (orc *)h;
  size_t N = (size_t)o->Ng;
  if (phi) memcpy(phi, o->phi, sizeof(double) * N);
  if (psi) memcpy(psi, o->psi, sizeof(double) * N);
  if (A) memcpy(A, o->A, sizeof(double) * 3 * N);
  if (U) memcpy(U, o->U, sizeof(double) * 3 * N);
  if (rho) memcpy(rho, o->rho, sizeof(double) * N);
  if (J) memcpy(J, o->J, sizeof(double) * 3 * N);
  return ORC_OK;
}

int orc_set_fields(void *h, const double *phi, const double *psi, const double *A,
                   const double *U, const double *rho, const double *J) {
  orc *o = (orc *)h;
  size_t N = (size_t)o->Ng;
  if (phi) memcpy(o->phi, phi, sizeof(double) * N);
  if (psi) memcpy(o->psi, psi, sizeof(double) * N);
  if (A) memcpy(o->A, A, sizeof(double) * 3 * N);
  if (U) memcpy(o->U, U, sizeof(double) * 3 * N);
  if (rho) memcpy(o->rho, rho, sizeof(double) * N);
  if (J) memcpy(o->J, J, sizeof(double) * 3 * N);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* knot-jump regularity diagnostic, Sec. 5.3                           */
/* ------------------------------------------------------------------ */
/* The field interpolants F_h(x) = sum_g F_g S(x - x_g) with the particle
   shape S of degree o->p.order, at the point u (node units, unwrapped):
   grad phi_h, U_h and grad A_h (columns per active dimension, physical
   units), from the B-spline formula on every node of a window of 6 nodes
   per active dimension around u (the support is 2 or 3 nodes wide). */
static void field_interp_at(const orc *o, const double u[3], double gphi[3], double Uh[3],
                            double gA[3][3]) {
  const int d = o->p.dim;
  const size_t Ng = (size_t)o->Ng;
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int l = 0; l < 3; l++) {
    gphi[l] = Uh[l] = 0.0;
    for (int j = 0; j < 3; j++) gA[l][j] = 0.0;
    if (l < d) {
      lo[l] = (int)floor(u[l]) - 2;
      hi[l] = lo[l] + 5;
    }
  }
  for (int m2 = lo[2]; m2 <= hi[2]; m2++)
    for (int m1 = lo[1]; m1 <= hi[1]; m1++)
      for (int m0 = lo[0]; m0 <= hi[0]; m0++) {
        const int m[3] = {m0, m1, m2};
        double S[3] = {1.0, 1.0, 1.0}, dS[3] = {0.0, 0.0, 0.0};
        size_t g = 0, stride = 1;
        for (int l = 0; l < d; l++) {
          const double xi = u[l] - m[l];
          S[l] = shp(o, xi);
          dS[l] = dshp(o, xi) / o->dx[l];
          const int n = o->p.n[l];
          g += stride * (size_t)(((m[l] % n) + n) % n);
          stride *= (size_t)n;
        }
        const double W = S[0] * S[1] * S[2];
        for (int c = 0; c < 3; c++) Uh[c] += o->U[c * Ng + g] * W;
        for (int l = 0; l < d; l++) {
          double Wd = dS[l];
          for (int q = 0; q < d; q++)
            if (q != l) Wd *= S[q];
          gphi[l] += o->phi[g] * Wd;
          for (int c = 0; c < 3; c++) gA[c][l] += o->A[c * Ng + g] * Wd;
        }
      }
}

/* For every active axis a and every node, the knot of the interpolant that
   follows the node along a (half a cell on for S_2, the node itself for
   S_1) is probed at +-eps (node units) along a.  The other coordinates sit
   half a cell away from their own knots (on the node for S_2, at the cell
   centre for S_1), where the interpolant is smooth in them.  The jumps are
   |E(+) - E(-)| of E_shape = -grad phi_h - U_h (Euclidean norm) and
   |G(+) - G(-)| of G = grad A_h (Frobenius norm); returns their maxima. */
int orc_knot_jumps(void *h, double eps, double *E_jump, double *G_jump) {
  orc *o = (orc *)h;
  const int d = o->p.dim;
  double Emax = 0.0, Gmax = 0.0;
  for (int a = 0; a < d; a++)
    for (long g = 0; g < o->Ng; g++) {
      long r = g;
      double u[3] = {0.0, 0.0, 0.0};
      const double side_off = o->p.order == 1 ? 0.5 : 0.0;  // transverse: off the knots
      for (int l = 0; l < d; l++) {
        u[l] = (double)(r % o->p.n[l]) + (l == a ? 0.0 : side_off);
        r /= o->p.n[l];
      }
      double E[2][3], G[2][3][3];
      for (int side = 0; side < 2; side++) {
        double up[3] = {u[0], u[1], u[2]}, gphi[3], Uh[3];
        up[a] += knot_off(o) + (side ? eps : -eps);
        field_interp_at(o, up, gphi, Uh, G[side]);
        for (int c = 0; c < 3; c++) E[side][c] = -(c < d ? gphi[c] : 0.0) - Uh[c];
      }
      double e2 = 0.0, g2 = 0.0;
      for (int c = 0; c < 3; c++) {
        e2 += (E[1][c] - E[0][c]) * (E[1][c] - E[0][c]);
        for (int l = 0; l < d; l++) g2 += (G[1][c][l] - G[0][c][l]) * (G[1][c][l] - G[0][c][l]);
      }
      if (sqrt(e2) > Emax) Emax = sqrt(e2);
      if (sqrt(g2) > Gmax) Gmax = sqrt(g2);
    }
  *E_jump = Emax;
  *G_jump = Gmax;
  return ORC_OK;
}

int orc_set_state(void *h, long np, const int *species, const double *x, const double *P,
                  const double *w, const double *phi, const double *psi, const double *A,
                  const double *U, const double *rho, const double *J) {
  orc *o = (orc *)h;
  int st = orc_set_particles(h, np, species, x, P, 1, w);
  if (st) return st;
  orc_set_fields(h, phi, psi, A, U, rho, J);
  o->pending_mech = 0;
  o->started = 1;
  return ORC_OK;
}

static double pq(const orc *o, long i) { return o->w[i] * o->p.q[o->sp[i]]; }
static double pm(const orc *o, long i) { return o->w[i] * o->p.m[o->sp[i]]; }

static void particle_x(const orc *o, long i, double *xp) {
  for (int l = 0; l < 3; l++) xp[l] = (l < o->p.dim) ? o->x[(size_t)l * o->np + i] : 0.0;
}

/* kinetic energy sum_i m kappa^2 (gamma(p_i) - 1) with p = P - q A_h(x),
   Eqs. Kkin-nondim, mechanical-endpoints-energy */
static double kinetic_energy(const orc *o) {
  double K = 0.0;
  size_t n = (size_t)o->np;
  for (size_t i = 0; i < n; i++) {
    double xp[3], u[3], Ax[3], p[3];
    particle_x(o, (long)i, xp);
    node_coord(o, xp, u);
    interp_point(o, u, o->A, 3, Ax);
    double q = pq(o, (long)i), m = pm(o, (long)i), k2 = o->p.kappa * o->p.kappa;
    for (int c = 0; c < 3; c++) p[c] = o->P[c * n + i] - q * Ax[c];
    double gam = sqrt(1.0 + dot3(p, p) / (m * m * k2));
    K += m * k2 * (gam - 1.0);
  }
  return K;
}

/* point deposits rho = sum q S(x)/dV + rho_bg and J = sum q v S(x)/dV */
static void point_deposit(orc *o, double *rho, double *J) {
  size_t n = (size_t)o->np, Ng = (size_t)o->Ng;
  int d = o->p.dim;
  for (size_t g = 0; g < Ng; g++) rho[g] = o->p.rho_bg;
  memset(J, 0, sizeof(double) * 3 * Ng);
  for (size_t i = 0; i < n; i++) {
    double xp[3], u[3], Ax[3], p[3], v[3];
    particle_x(o, (long)i, xp);
    node_coord(o, xp, u);
    interp_point(o, u, o->A, 3, Ax);
    double q = pq(o, (long)i), m = pm(o, (long)i), k2 = o->p.kappa * o->p.kappa;
    for (int c = 0; c < 3; c++) p[c] = o->P[c * n + i] - q * Ax[c];
    double gam = sqrt(1.0 + dot3(p, p) / (m * m * k2));
    for (int c = 0; c < 3; c++) v[c] = p[c] / (m * gam);
    int lo[3] = {0, 0, 0}, wn[3] = {1, 1, 1};
    for (int l = 0; l < d; l++) {
      lo[l] = (int)floor(u[l] - shp_rad(o));
      wn[l] = (int)ceil(u[l] + shp_rad(o)) - lo[l] + 1;
    }
    for (int c2 = 0; c2 < wn[2]; c2++)
      for (int c1 = 0; c1 < wn[1]; c1++)
        for (int c0 = 0; c0 < wn[0]; c0++) {
          int cc[3] = {c0, c1, c2}, gi[3] = {0, 0, 0};
          double S = 1.0;
          for (int l = 0; l < d; l++) {
            S *= shp(o, u[l] - (lo[l] + cc[l]));
            gi[l] = mod(lo[l] + cc[l], o->p.n[l]);
          }
          size_t g = (size_t)gi[0] + (size_t)o->p.n[0] * (gi[1] + (size_t)o->p.n[1] * gi[2]);
          rho[g] += q * S / o->dV;
          for (int c = 0; c < 3; c++) J[c * Ng + g] += q * v[c] * S / o->dV;
        }
  }
}

int orc_start(void *h, orc_report *rep) {
  orc *o = (orc *)h;
  size_t n = (size_t)o->np, Ng = (size_t)o->Ng;
  double k2c = o->p.kappa * o->p.kappa;
  orc_project(o, o->A, 3);
  orc_project(o, o->U, 3);
  if (o->pending_mech) { /* P = m u + q (P A)_h(x), Sec. 4.5 Nyquist paragraph */
    for (size_t i = 0; i < n; i++) {
      double xp[3], u[3], Ax[3];
      particle_x(o, (long)i, xp);
      node_coord(o, xp, u);
      interp_point(o, u, o->A, 3, Ax);
      for (int c = 0; c < 3; c++)
        o->P[c * n + i] = pm(o, (long)i) * o->u_mech[c * n + i] + pq(o, (long)i) * Ax[c];
    }
    o->pending_mech = 0;
  }
  point_deposit(o, o->rho, o->J);
  orc_project(o, o->rho, 1);
  orc_project(o, o->J, 3);
  /* Gauss: -Lap phi = sigma1 rho + div U ; Lorenz: psi = -kappa^2 div A */
  double complex *rh = cbuf(o), *Ph = cbuf(o), *Qh = cbuf(o), *Uh[3], *Ah[3];
  fwd(o, o->rho, rh);
  for (int a = 0; a < 3; a++) {
    Uh[a] = cbuf(o); Ah[a] = cbuf(o);
    fwd(o, o->U + a * Ng, Uh[a]);
    fwd(o, o->A + a * Ng, Ah[a]);
  }
  for (size_t g = 0; g < Ng; g++) {
    double kt[3]; int nq;
    mode_of(o, (int)g, kt, &nq);
    double kk = kt[0] * kt[0] + kt[1] * kt[1] + kt[2] * kt[2];
    double complex divU = I * (kt[0] * Uh[0][g] + kt[1] * Uh[1][g] + kt[2] * Uh[2][g]);
    double complex divA = I * (kt[0] * Ah[0][g] + kt[1] * Ah[1][g] + kt[2] * Ah[2][g]);
    Ph[g] = (kk > 0.0 && !(nq && o->p.project)) ? (o->p.sigma1 * rh[g] + divU) / kk : 0.0;
    Qh[g] = (nq && o->p.project) ? 0.0 : -k2c * divA;
  }
  inv(o, Ph, o->phi);
  inv(o, Qh, o->psi);
  for (int a = 0; a < 3; a++) { free(Uh[a]); free(Ah[a]); }
  free(rh); free(Ph); free(Qh);
  double K = kinetic_energy(o);
  double W = orc_field_energy(o, o->phi, o->A, o->U);
  o->E0 = K + W;
  o->started = 1;
  if (rep) {
    memset(rep, 0, sizeof *rep);
    rep->K = K; rep->W = W; rep->E_tot = K + W;
    orc_constraint_rms(o, o->phi, o->psi, o->A, o->U, o->rho, &rep->gauss_rms,
                       &rep->lorenz_rms);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* map evaluation H(j) = P J_orb(j), Sec. 4.5                          */
/* ------------------------------------------------------------------ */
typedef struct {
  double *gradphi, *A1, *Uh, *phi1, *psi1, *U1, *rho1; /* field-solve outputs */
  double *Jorb;
  double work_particles, chain_sq; /* final-pass sums */
} eval_t;

static void eval_alloc(const orc *o, eval_t *e) {
  size_t N = (size_t)o->Ng;
  e->gradphi = (double *)calloc(3 * N, sizeof(double));
  e->A1 = (double *)calloc(3 * N, sizeof(double));
  e->Uh = (double *)calloc(3 * N, sizeof(double));
  e->U1 = (double *)calloc(3 * N, sizeof(double));
  e->phi1 = (double *)calloc(N, sizeof(double));
  e->psi1 = (double *)calloc(N, sizeof(double));
  e->rho1 = (double *)calloc(N, sizeof(double));
  e->Jorb = (double *)calloc(3 * N, sizeof(double));
}

static void eval_free(eval_t *e) {
  free(e->gradphi); free(e->A1); free(e->Uh); free(e->U1);
  free(e->phi1); free(e->psi1); free(e->rho1); free(e->Jorb);
}

/* step start: A^- = A^n_h(x^n), p^n = P^n - q A^-, v^0 = p^n / (m gamma(p^n)) */
static void step_start(orc *o) {
  size_t n = (size_t)o->np;
  for (size_t i = 0; i < n; i++) {
    double xp[3], u[3], Ax[3];
    particle_x(o, (long)i, xp);
    node_coord(o, xp, u);
    interp_point(o, u, o->A, 3, Ax);
    double q = pq(o, (long)i), m = pm(o, (long)i);
    double p[3];
    for (int c = 0; c < 3; c++) {
      o->Am[c * n + i] = Ax[c];
      p[c] = o->P[c * n + i] - q * Ax[c];
      o->pn[c * n + i] = p[c];
    }
    double gam = sqrt(1.0 + dot3(p, p) / (m * m * o->p.kappa * o->p.kappa));
    for (int c = 0; c < 3; c++) o->v0[c * n + i] = p[c] / (m * gam);
  }
}

/* ------------------------------------------------------------------ */
/* one particle's inner solve (Sec. 4.5) with convergence-triggered    */
/* refinement (Sec. 5.3, reading R16)                                  */
/* ------------------------------------------------------------------ */

/* time levels s_k = k / 2^R of the field step and the mesh potentials
   A(s_k) = (1 - s_k) A^n + s_k A^{n+1} there (Eq. A-g-s) */
typedef struct {
  int R, nlev;
  const double *A[(1 << REFMAX) + 1];
  double *own[(1 << REFMAX) + 1];
} tlev_t;

static void tlev_make(const orc *o, const double *An, const double *A1, tlev_t *t) {
  int R = o->p.refine_max < 0 ? 0 : (o->p.refine_max > REFMAX ? REFMAX : o->p.refine_max);
  size_t N3 = (size_t)3 * o->Ng;
  t->R = R;
  t->nlev = (1 << R) + 1;
  for (int k = 0; k < t->nlev; k++) {
    t->own[k] = NULL;
    if (k == 0) { t->A[k] = An; continue; }
    if (k == t->nlev - 1) { t->A[k] = A1; continue; }
    double sk = (double)k / (double)(1 << R);
    double *a = (double *)malloc(sizeof(double) * N3);
    for (size_t q = 0; q < N3; q++) a[q] = (1.0 - sk) * An[q] + sk * A1[q];
    t->own[k] = a;
    t->A[k] = a;
  }
}

static void tlev_free(tlev_t *t) {
  for (int k = 0; k < t->nlev; k++) free(t->own[k]);
}

typedef struct {
  int nsub, stride;                 /* substeps of the accepted level, level-table stride */
  double xs[1 << REFMAX][3];        /* start position of each substep */
  double vb[1 << REFMAX][3];        /* converged orbit velocity of each substep */
  double Pnew[3], vbar[3];          /* P^{n+1}; orbit velocity averaged over the substeps */
  int iters;                        /* Picard iterations of the accepted level */
} psolve_t;

/* Level 0 is one particle step over the whole field step.  If any Picard
   iteration fails (limit, non-finite or superluminal velocity, orbit wider
   than the node window), level L retries with 2^L equal substeps, each
   converged in turn from the previous substep's end state.  Returns 1 on
   success; on failure ps holds the last iterate of level 0. */
static int solve_particle(const orc *o, long i, const double *gradphi, const tlev_t *tl,
                          double tau_r, double tau_a, psolve_t *ps) {
  size_t n = (size_t)o->np;
  double q = pq(o, i), m = pm(o, i), kap = o->p.kappa;
  double x0[3], P0[3];
  particle_x(o, i, x0);
  for (int c = 0; c < 3; c++) P0[c] = o->P[c * n + i];
  for (int lvl = 0; lvl <= tl->R; lvl++) {
    int nsub = 1 << lvl, stride = 1 << (tl->R - lvl);
    double dtau = o->p.dt / nsub;
    double x[3] = {x0[0], x0[1], x0[2]}, P[3] = {P0[0], P0[1], P0[2]};
    int ok = 1, its = 0;
    for (int sub = 0; sub < nsub && ok; sub++) {
      const double *Aa = tl->A[sub * stride], *Ab = tl->A[(sub + 1) * stride];
      double u[3], Am[3], p[3], vb[3], Pk[3];
      node_coord(o, x, u);
      interp_point(o, u, Aa, 3, Am);
      for (int c = 0; c < 3; c++) p[c] = P[c] - q * Am[c];
      double gam = sqrt(1.0 + dot3(p, p) / (m * m * kap * kap));
      for (int c = 0; c < 3; c++) {
        vb[c] = p[c] / (m * gam); /* reading R5 */
        Pk[c] = P[c];
      }
      int conv = 0;
      orbit_t ob;
      for (int it = 1; it <= o->p.inner_max; it++) {
        its++;
        if (orbit_eval(o, x, vb, dtau, gradphi, Aa, Ab, NULL, &ob, 0)) break;
        double pmn[3], ppl[3], Pn1[3], vn[3];
        orc_push(P, Am, ob.Aplus, ob.gphi, ob.D, vb, q, m, kap, dtau, pmn, ppl, Pn1, vn);
        double diff = 0.0, nrm = 0.0;
        int finite = 1;
        for (int c = 0; c < 3; c++) {
          if (!isfinite(vn[c])) finite = 0;
          diff = fmax(diff, fabs(vn[c] - vb[c]));
          nrm = fmax(nrm, fabs(vn[c]));
        }
        if (!finite || sqrt(dot3(vn, vn)) >= kap) break;
        for (int c = 0; c < 3; c++) {
          vb[c] = vn[c];
          Pk[c] = Pn1[c];
        }
        if (diff <= tau_a + tau_r * nrm) { conv = 1; break; }
      }
      if (lvl == 0) { /* report the level-0 iterate if every level fails */
        for (int c = 0; c < 3; c++) { ps->vbar[c] = vb[c]; ps->Pnew[c] = Pk[c]; }
      }
      if (!conv) { ok = 0; break; }
      for (int c = 0; c < 3; c++) {
        ps->xs[sub][c] = x[c];
        ps->vb[sub][c] = vb[c];
      }
      for (int l = 0; l < o->p.dim; l++) x[l] += dtau * vb[l];
      for (int c = 0; c < 3; c++) P[c] = Pk[c];
    }
    if (ok) {
      ps->nsub = nsub;
      ps->stride = stride;
      ps->iters = its;
      for (int c = 0; c < 3; c++) {
        double v = 0.0;
        for (int sub = 0; sub < nsub; sub++) v += ps->vb[sub][c];
        ps->vbar[c] = v / nsub;
        ps->Pnew[c] = P[c];
      }
      return 1;
    }
  }
  ps->nsub = 0;
  ps->iters = -1;
  return 0;
}

/* one map evaluation at trial current j; returns 0 or ORC_EINNER */
static int map_eval(orc *o, const double *j, double tau_r, double tau_a, eval_t *e,
                    double *H, int final_pass) {
  size_t n = (size_t)o->np, Ng = (size_t)o->Ng;
  double *jp = (double *)malloc(sizeof(double) * 3 * Ng);
  memcpy(jp, j, sizeof(double) * 3 * Ng);
  orc_project(o, jp, 3);
  orc_field_solve(o, jp, e->gradphi, e->A1, e->Uh, e->phi1, e->psi1, e->U1, e->rho1);
  free(jp);
  int fail = 0;
  long refined = 0;
  tlev_t tl;
  tlev_make(o, o->A, e->A1, &tl);
#pragma omp parallel for schedule(dynamic, 64) reduction(| : fail) reduction(+ : refined)
  for (long i = 0; i < (long)n; i++) {
    psolve_t ps;
    int conv = solve_particle(o, i, e->gradphi, &tl, tau_r, tau_a, &ps);
    o->iters[i] = ps.iters;
    o->nsub[i] = ps.nsub;
    for (int c = 0; c < 3; c++) {
      o->vbar[c * n + i] = ps.vbar[c];
      o->Pnew[c * n + i] = ps.Pnew[c];
    }
    if (ps.nsub > 1) refined++;
    if (!conv) fail |= 1;
  }
  o->refined = refined;
  if (fail) {
    tlev_free(&tl);
    return ORC_EINNER;
  }
  /* deposit with the final orbit velocity, Eq. orbit-current-energy; the
     same pass evaluates the chain-rule and work sums of Sec. 4.4 */
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  double *part = (double *)calloc((size_t)nthr * 3 * Ng, sizeof(double));
  double work = 0.0, chain = 0.0;
#pragma omp parallel reduction(+ : work, chain)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    double *Jt = part + (size_t)t * 3 * Ng;
#pragma omp for schedule(static)
    for (long i = 0; i < (long)n; i++) {
      psolve_t ps;
      if (o->nsub[i] > 1) {
        /* refined particle: recover its substeps (deterministic re-solve) */
        solve_particle(o, i, e->gradphi, &tl, tau_r, tau_a, &ps);
      } else {
        ps.nsub = 1;
        ps.stride = 1 << tl.R;
        particle_x(o, i, ps.xs[0]);
        for (int c = 0; c < 3; c++) ps.vb[0][c] = o->vbar[c * n + i];
      }
      double q = pq(o, i), wsub = 1.0 / ps.nsub, dtau = o->p.dt / ps.nsub;
      for (int sub = 0; sub < ps.nsub; sub++) {
        const double *Aa = tl.A[sub * ps.stride], *Ab = tl.A[(sub + 1) * ps.stride];
        const double *vb = ps.vb[sub];
        orbit_t ob;
        orbit_eval(o, ps.xs[sub], vb, dtau, e->gradphi, Aa, Ab, e->Uh, &ob, 1);
        /* orbit-averaged current: each substep weighs its share of the step */
        for (int c2 = 0; c2 < ob.wn[2]; c2++)
          for (int c1 = 0; c1 < ob.wn[1]; c1++)
            for (int c0 = 0; c0 < ob.wn[0]; c0++) {
              int cc[3] = {c0, c1, c2}, gi[3];
              for (int l = 0; l < 3; l++) gi[l] = mod(ob.lo[l] + cc[l], o->p.n[l]);
              size_t g = (size_t)gi[0] + (size_t)o->p.n[0] * (gi[1] + (size_t)o->p.n[1] * gi[2]);
              double Sb = ob.Sbar[c0 + ob.wn[0] * (c1 + ob.wn[1] * c2)];
              for (int c = 0; c < 3; c++) Jt[c * Ng + g] += wsub * q * vb[c] * Sb / o->dV;
            }
        if (final_pass) {
          double Dv[3], Am[3], u[3];
          node_coord(o, ps.xs[sub], u);
          interp_point(o, u, Aa, 3, Am);
          for (int c = 0; c < 3; c++)
            Dv[c] = ob.D[c * 3 + 0] * vb[0] + ob.D[c * 3 + 1] * vb[1] + ob.D[c * 3 + 2] * vb[2];
          for (int c = 0; c < 3; c++) {
            double Ebar = -ob.gphi[c] - ob.Ubar[c];
            work += wsub * q * vb[c] * Ebar;
            double RA = ob.Aplus[c] - Am[c] - dtau * (ob.Ubar[c] + Dv[c]);
            chain += RA * RA;
          }
        }
      }
    }
  }
  memset(e->Jorb, 0, sizeof(double) * 3 * Ng);
  for (int t = 0; t < nthr; t++)
    for (size_t k = 0; k < 3 * Ng; k++) e->Jorb[k] += part[(size_t)t * 3 * Ng + k];
  free(part);
  tlev_free(&tl);
  e->work_particles = work;
  e->chain_sq = chain;
  memcpy(H, e->Jorb, sizeof(double) * 3 * Ng);
  orc_project(o, H, 3);
  return ORC_OK;
}

int orc_deposit(void *h, const double *vbar, double *Jorb) {
  orc *o = (orc *)h;
  size_t n = (size_t)o->np, Ng = (size_t)o->Ng;
  double *zero = (double *)calloc(3 * Ng, sizeof(double));
  memset(Jorb, 0, sizeof(double) * 3 * Ng);
  for (size_t i = 0; i < n; i++) {
    double xp[3], vb[3];
    particle_x(o, (long)i, xp);
    for (int c = 0; c < 3; c++) vb[c] = vbar[c * n + i];
    orbit_t ob;
    if (orbit_eval(o, xp, vb, o->p.dt, NULL, zero, zero, NULL, &ob, 1)) {
      free(zero);
      return ORC_EARG;
    }
    for (int c2 = 0; c2 < ob.wn[2]; c2++)
      for (int c1 = 0; c1 < ob.wn[1]; c1++)
        for (int c0 = 0; c0 < ob.wn[0]; c0++) {
          int cc[3] = {c0, c1, c2}, gi[3];
          for (int l = 0; l < 3; l++) gi[l] = mod(ob.lo[l] + cc[l], o->p.n[l]);
          size_t g = (size_t)gi[0] + (size_t)o->p.n[0] * (gi[1] + (size_t)o->p.n[1] * gi[2]);
          double Sb = ob.Sbar[c0 + ob.wn[0] * (c1 + ob.wn[1] * c2)];
          for (int c = 0; c < 3; c++) Jorb[c * Ng + g] += pq(o, (long)i) * vb[c] * Sb / o->dV;
        }
  }
  free(zero);
  return ORC_OK;
}

int orc_orbit_data(void *h, const double *x, const double *vbar, const double *gradphi,
                   const double *An, const double *Anp1, const double *Uhalf, double *gphi,
                   double *Ubar, double *D, double *Aplus, double *Aminus, double *Sbar_sum) {
  orc *o = (orc *)h;
  orbit_t ob;
  double xp[3] = {0, 0, 0};
  for (int l = 0; l < o->p.dim; l++) xp[l] = x[l];
  if (orbit_eval(o, xp, vbar, o->p.dt, gradphi, An, Anp1, Uhalf, &ob, 1)) return ORC_EARG;
  for (int c = 0; c < 3; c++) {
    if (gphi) gphi[c] = ob.gphi[c];
    if (Ubar) Ubar[c] = ob.Ubar[c];
    if (Aplus) Aplus[c] = ob.Aplus[c];
  }
  if (D) memcpy(D, ob.D, sizeof ob.D);
  if (Aminus) {
    double u[3];
    node_coord(o, xp, u);
    interp_point(o, u, An, 3, Aminus);
  }
  if (Sbar_sum) *Sbar_sum = ob.Sbar_sum;
  return ORC_OK;
}

int orc_eval_map(void *h, const double *j, double tol, double *H, double *vbar,
                 double *Pnew, int *inner_counts) {
  orc *o = (orc *)h;
  size_t n = (size_t)o->np;
  step_start(o);
  eval_t e;
  eval_alloc(o, &e);
  double *Hb = (double *)malloc(sizeof(double) * 3 * o->Ng);
  double ti = tol * o->p.inner_tol_scale;
  int st = map_eval(o, j, ti, ti * o->p.tol_abs_ratio, &e, Hb, 0);
  if (H) memcpy(H, Hb, sizeof(double) * 3 * o->Ng);
  if (vbar) memcpy(vbar, o->vbar, sizeof(double) * 3 * n);
  if (Pnew) memcpy(Pnew, o->Pnew, sizeof(double) * 3 * n);
  if (inner_counts) memcpy(inner_counts, o->iters, sizeof(int) * n);
  free(Hb);
  eval_free(&e);
  return st;
}

/* ------------------------------------------------------------------ */
/* outer acceptance tests, Eq. mixed-nonlinear-tests                  */
/* ------------------------------------------------------------------ */
static double rms_n(size_t N3, const double *v) {
  double s = 0.0;
  for (size_t k = 0; k < N3; k++) s += v[k] * v[k];
  return sqrt(s / (double)N3);
}

/* Eq. mixed-nonlinear-tests: the scaled RMS test and the scaled maximum-node
   test.  Ng nodes, 3 components per node stored component-major (c*Ng + g);
   |.| of a node is the Euclidean norm of its 3 components. */
void orc_scaled_tests(long Ng_l, const double *r, const double *H, const double *j,
                      double tau_r, double tau_a, double *srms, double *smax) {
  size_t Ng = (size_t)Ng_l, N3 = 3 * Ng;
  *srms = rms_n(N3, r) / (tau_a + 0.5 * tau_r * (rms_n(N3, H) + rms_n(N3, j)));
  double mx = 0.0;
  for (size_t g = 0; g < Ng; g++) {
    double rr = 0.0, hh = 0.0, jj = 0.0;
    for (int c = 0; c < 3; c++) {
      rr += r[c * Ng + g] * r[c * Ng + g];
      hh += H[c * Ng + g] * H[c * Ng + g];
      jj += j[c * Ng + g] * j[c * Ng + g];
    }
    double v = sqrt(rr) / (tau_a + 0.5 * tau_r * (sqrt(hh) + sqrt(jj)));
    if (v > mx) mx = v;
  }
  *smax = mx;
}

/* Gaussian elimination with partial pivoting for the small Anderson system */
static int small_solve(int m, double *Amat, double *b) {
  for (int c = 0; c < m; c++) {
    int piv = c;
    for (int r = c + 1; r < m; r++)
      if (fabs(Amat[r * m + c]) > fabs(Amat[piv * m + c])) piv = r;
    if (Amat[piv * m + c] == 0.0) return -1;
    if (piv != c) {
      for (int k = 0; k < m; k++) {
        double t = Amat[c * m + k]; Amat[c * m + k] = Amat[piv * m + k]; Amat[piv * m + k] = t;
      }
      double t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    for (int r = c + 1; r < m; r++) {
      double f = Amat[r * m + c] / Amat[c * m + c];
      for (int k = c; k < m; k++) Amat[r * m + k] -= f * Amat[c * m + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = m - 1; c >= 0; c--) {
    double s = b[c];
    for (int k = c + 1; k < m; k++) s -= Amat[c * m + k] * b[k];
    b[c] = s / Amat[c * m + c];
    if (!isfinite(b[c])) return -1;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* the outer solve of Algorithm 1 on a map H(j) given as a callback   */
/* ------------------------------------------------------------------ */
/* map(user, j, H, final_pass): H = H(j); returns ORC_OK or ORC_EINNER */
typedef int (*outer_map_fn)(void *user, const double *j, double *H, int final_pass);

static void trace_put(orc_outer_trace *tr, int k, const double *j, size_t N3, double srms,
                      double smax) {
  if (!tr || k >= tr->cap) return;
  if (tr->j) memcpy(tr->j + (size_t)k * N3, j, sizeof(double) * N3);
  if (tr->srms) tr->srms[k] = srms;
  if (tr->smax) tr->smax[k] = smax;
  if (tr->kind) tr->kind[k] = -1;
  if (tr->alpha) tr->alpha[k] = 0.0;
  if (tr->mh) tr->mh[k] = 0;
  tr->n = k + 1;
}

/* Converges H(j) = j from the trial current j (Algorithm 1): at every outer
   iteration the tests of Eq. mixed-nonlinear-tests; when both pass, one more
   evaluation at the same j (final_pass = 1) that must pass them again;
   otherwise a direction, type-II Anderson (Eq. anderson-type-two-update) once
   the iteration is eligible and history exists, else damped Picard beta r,
   with backtracking alpha = 1, 1/2, .. (backtrack_levels values) under the
   sufficient-decrease and maximum-node safeguards; a rejected Anderson
   direction is retried as damped Picard.  The accepted trial's evaluation
   gives the next iterate's H(j).  History: the differences of successive
   accepted (j, r), at most anderson_m columns (oldest dropped), cleared when
   the regularised Gram system has no finite solution or when the RMS
   residual grows by more than growth_limit (reading R8; growth_scaled
   selects the scaled RMS of Eq. mixed-nonlinear-tests instead of the plain
   RMS).  On return j holds the last iterate and H its map value (the
   verification's, on success).  R receives outer_iters (the iterations
   begun, counting the one whose tests pass), map_evals and the scaled
   residuals. */
static int outer_solve(const orc_params *p, size_t Ng, outer_map_fn map, void *user,
                       double tau_r, double tau_a, double *j, double *H, orc_report *R,
                       orc_outer_trace *tr) {
  size_t N3 = 3 * Ng;
  int M = p->anderson_m;
  double *r = (double *)malloc(sizeof(double) * N3);
  double *jt = (double *)malloc(sizeof(double) * N3);
  double *Ht = (double *)malloc(sizeof(double) * N3);
  double *rt = (double *)malloc(sizeof(double) * N3);
  double *dir = (double *)malloc(sizeof(double) * N3);
  double *dJ = (double *)calloc((size_t)(M > 0 ? M : 1) * N3, sizeof(double));
  double *dR = (double *)calloc((size_t)(M > 0 ? M : 1) * N3, sizeof(double));
  int mh = 0;
  if (tr) tr->n = 0;
  int status = map(user, j, H, 0);
  R->map_evals = 1;
  for (size_t q = 0; q < N3; q++) r[q] = H[q] - j[q];
  int done = 0;
  for (int k = 0; status == ORC_OK && k < p->outer_max; k++) {
    double srms, smax;
    orc_scaled_tests((long)Ng, r, H, j, tau_r, tau_a, &srms, &smax);
    R->outer_iters = k + 1;
    R->res_scaled_rms = srms;
    R->res_scaled_max = smax;
    trace_put(tr, k, j, N3, srms, smax);
    if (srms <= 1.0 && smax <= 1.0) {
      /* verify by re-evaluating the map at the candidate current */
      status = map(user, j, H, 1);
      R->map_evals++;
      if (status != ORC_OK) break;
      for (size_t q = 0; q < N3; q++) r[q] = H[q] - j[q];
      orc_scaled_tests((long)Ng, r, H, j, tau_r, tau_a, &srms, &smax);
      R->res_scaled_rms = srms;
      R->res_scaled_max = smax;
      if (!(srms <= 1.0 && smax <= 1.0)) { status = ORC_EOUTER; break; }
      done = 1;
      break;
    }
    /* proposed directions: Anderson (type II) when eligible, else Picard */
    int have_anderson = 0;
    if (k + 1 >= p->anderson_start && mh > 0) {  /* iterations counted from 1 */
      double G[ORC_MAX_ANDERSON * ORC_MAX_ANDERSON], b[ORC_MAX_ANDERSON], trg = 0.0;
      for (int a = 0; a < mh; a++) {
        for (int c = 0; c < mh; c++) {
          double s = 0.0;
          for (size_t q = 0; q < N3; q++) s += dR[a * N3 + q] * dR[c * N3 + q];
          G[a * mh + c] = s;
        }
        double s = 0.0;
        for (size_t q = 0; q < N3; q++) s += dR[a * N3 + q] * r[q];
        b[a] = s;
        trg += G[a * mh + a];
      }
      for (int a = 0; a < mh; a++) G[a * mh + a] += p->lambda * trg / mh;
      if (isfinite(trg) && trg > 0.0 && small_solve(mh, G, b) == 0) {
        have_anderson = 1;
        for (size_t q = 0; q < N3; q++) {
          double s = p->beta * r[q];
          for (int a = 0; a < mh; a++) s -= (dJ[a * N3 + q] + p->beta * dR[a * N3 + q]) * b[a];
          dir[q] = s; /* j_A - j */
        }
      } else {
        mh = 0; /* unusable history */
      }
    }
    int accepted = 0, kind = 0;
    double alpha_ok = 0.0, srt = 0.0, smt = 0.0;
    for (int attempt = have_anderson ? 0 : 1; attempt < 2 && !accepted; attempt++) {
      if (attempt == 1)
        for (size_t q = 0; q < N3; q++) dir[q] = p->beta * r[q];
      double alpha = 1.0;
      for (int lvl = 0; lvl < p->backtrack_levels; lvl++, alpha *= 0.5) {
        for (size_t q = 0; q < N3; q++) jt[q] = j[q] + alpha * dir[q];
        status = map(user, jt, Ht, 0);
        R->map_evals++;
        if (status != ORC_OK) break;
        for (size_t q = 0; q < N3; q++) rt[q] = Ht[q] - jt[q];
        orc_scaled_tests((long)Ng, rt, Ht, jt, tau_r, tau_a, &srt, &smt);
        if (srt <= (1.0 - p->decrease_coef * alpha) * srms && smt <= p->growth_limit * smax) {
          accepted = 1;
          alpha_ok = alpha;
          kind = attempt == 0 ? 1 : (have_anderson ? 2 : 0);
          break;
        }
      }
      if (status != ORC_OK) break;
    }
    if (status != ORC_OK) break;
    if (!accepted) { status = ORC_EOUTER; break; }
    /* history update; cleared when the residual grew too much */
    if (M > 0) {
      if (mh == M) {
        memmove(dJ, dJ + N3, sizeof(double) * (size_t)(M - 1) * N3);
        memmove(dR, dR + N3, sizeof(double) * (size_t)(M - 1) * N3);
        mh--;
      }
      for (size_t q = 0; q < N3; q++) {
        dJ[mh * N3 + q] = jt[q] - j[q];
        dR[mh * N3 + q] = rt[q] - r[q];
      }
      mh++;
      double grown = p->growth_scaled ? srt / srms : rms_n(N3, rt) / rms_n(N3, r);
      if (grown > p->growth_limit) mh = 0;
    }
    if (tr && k < tr->cap) {
      if (tr->kind) tr->kind[k] = kind;
      if (tr->alpha) tr->alpha[k] = alpha_ok;
      if (tr->mh) tr->mh[k] = mh;
    }
    memcpy(j, jt, sizeof(double) * N3);
    memcpy(H, Ht, sizeof(double) * N3);
    memcpy(r, rt, sizeof(double) * N3);
  }
  if (status == ORC_OK && !done) status = ORC_EOUTER;
  free(r); free(jt); free(Ht); free(rt); free(dir); free(dJ); free(dR);
  return status;
}

/* the particle map of one step as the outer solve's callback */
typedef struct {
  orc *o;
  eval_t *e;
  double ti_r, ti_a;
} particle_map_t;

static int particle_map(void *user, const double *j, double *H, int final_pass) {
  particle_map_t *pm = (particle_map_t *)user;
  return map_eval(pm->o, j, pm->ti_r, pm->ti_a, pm->e, H, final_pass);
}

/* an affine stand-in map H(j) = M j + b (test support) */
typedef struct {
  size_t N3;
  const double *M, *b;
} affine_map_t;

static int affine_map(void *user, const double *j, double *H, int final_pass) {
  (void)final_pass;
  affine_map_t *am = (affine_map_t *)user;
  for (size_t a = 0; a < am->N3; a++) {
    double s = am->b[a];
    for (size_t c = 0; c < am->N3; c++) s += am->M[a * am->N3 + c] * j[c];
    H[a] = s;
  }
  return ORC_OK;
}

int orc_outer_affine(const orc_params *prm, long Ng, const double *M, const double *b,
                     double *j, double tol, orc_outer_trace *tr, orc_report *rep) {
  if (!prm || Ng < 1 || !M || !b || !j || prm->anderson_m < 0 ||
      prm->anderson_m > ORC_MAX_ANDERSON)
    return ORC_EARG;
  size_t N3 = 3 * (size_t)Ng;
  affine_map_t am = {N3, M, b};
  orc_report R;
  memset(&R, 0, sizeof R);
  double *H = (double *)malloc(sizeof(double) * N3);
  int st = outer_solve(prm, (size_t)Ng, affine_map, &am, tol, tol * prm->tol_abs_ratio, j, H, &R,
                       tr);
  free(H);
  R.status = st;
  if (rep) *rep = R;
  return st;
}

/* ------------------------------------------------------------------ */
/* one implicit step, Algorithm 1                                      */
/* ------------------------------------------------------------------ */
int orc_step(void *h, double tol, orc_report *rep) {
  orc *o = (orc *)h;
  if (!o->started) return ORC_EARG;
  size_t n = (size_t)o->np, Ng = (size_t)o->Ng, N3 = 3 * Ng;
  double tau_r = tol, tau_a = tol * o->p.tol_abs_ratio;
  double ti_r = tol * o->p.inner_tol_scale, ti_a = ti_r * o->p.tol_abs_ratio;
  orc_report R;
  memset(&R, 0, sizeof R);

  step_start(o);
  double *j = (double *)malloc(sizeof(double) * N3);
  double *H = (double *)malloc(sizeof(double) * N3);
  eval_t e;
  eval_alloc(o, &e);
  memcpy(j, o->J, sizeof(double) * N3);
  particle_map_t pm = {o, &e, ti_r, ti_a};
  int status = outer_solve(&o->p, Ng, particle_map, &pm, tau_r, tau_a, j, H, &R, NULL);

  if (status == ORC_OK) {
    /* commit: x^{n+1} = x^n + dt vbar, P^{n+1}, fields at n+1, J^{n+1/2} */
    for (size_t i = 0; i < n; i++) {
      for (int l = 0; l < o->p.dim; l++)
        o->x[l * n + i] = wrap_pos(o, l, o->x[l * n + i] + o->p.dt * o->vbar[l * n + i]);
      for (int c = 0; c < 3; c++) o->P[c * n + i] = o->Pnew[c * n + i];
    }
    /* work residual, Eq. work-diagnostic, before the fields are replaced */
    double mesh_work = 0.0;
    for (size_t g = 0; g < Ng; g++)
      for (int c = 0; c < 3; c++) {
        double Eh = -e.gradphi[c * Ng + g] - e.Uh[c * Ng + g];
        mesh_work += e.Jorb[c * Ng + g] * Eh * o->dV;
      }
    R.work_residual = o->p.dt * (e.work_particles - mesh_work);
    R.chain_rms = n ? sqrt(e.chain_sq / (3.0 * n)) : 0.0;
    memcpy(o->phi, e.phi1, sizeof(double) * Ng);
    memcpy(o->psi, e.psi1, sizeof(double) * Ng);
    memcpy(o->rho, e.rho1, sizeof(double) * Ng);
    memcpy(o->A, e.A1, sizeof(double) * N3);
    memcpy(o->U, e.U1, sizeof(double) * N3);
    {
      double *jp = (double *)malloc(sizeof(double) * N3);
      memcpy(jp, j, sizeof(double) * N3);
      orc_project(o, jp, 3);
      memcpy(o->J, jp, sizeof(double) * N3);
      free(jp);
    }
    R.K = kinetic_energy(o);
    R.W = orc_field_energy(o, o->phi, o->A, o->U);
    R.E_tot = R.K + R.W;
    R.rel_dE = (R.E_tot - o->E0) / o->E0;
    orc_constraint_rms(o, o->phi, o->psi, o->A, o->U, o->rho, &R.gauss_rms, &R.lorenz_rms);
    long s = 0; int mx = 0;
    for (size_t i = 0; i < n; i++) { s += o->iters[i]; if (o->iters[i] > mx) mx = o->iters[i]; }
    R.inner_mean = n ? (double)s / n : 0.0;
    R.inner_max = mx;
  }
  R.status = status;
  if (rep) *rep = R;
  eval_free(&e);
  free(j); free(H);
  return status;
}

/* ------------------------------------------------------------------ */
/* inner solves of a subset of particles at trial current j (Sec. 4.5: */
/* with the trial fields fixed, every particle's orbit is converged    */
/* independently), for checks at sizes where a full evaluation is slow */
/* ------------------------------------------------------------------ */
int orc_eval_particles(void *h, const double *j, double tol, long nidx, const long *idx,
                       double *vbar, double *Pnew, int *inner_counts) {
  orc *o = (orc *)h;
  size_t Ng = (size_t)o->Ng;
  double ti = tol * o->p.inner_tol_scale, ta = ti * o->p.tol_abs_ratio;
  double *jp = (double *)malloc(sizeof(double) * 3 * Ng);
  memcpy(jp, j, sizeof(double) * 3 * Ng);
  orc_project(o, jp, 3);
  eval_t e;
  eval_alloc(o, &e);
  orc_field_solve(o, jp, e.gradphi, e.A1, e.Uh, e.phi1, e.psi1, e.U1, e.rho1);
  free(jp);
  int fail = 0;
  tlev_t tl;
  tlev_make(o, o->A, e.A1, &tl);
#pragma omp parallel for schedule(dynamic, 16) reduction(| : fail)
  for (long k = 0; k < nidx; k++) {
    psolve_t ps;
    int conv = solve_particle(o, idx[k], e.gradphi, &tl, ti, ta, &ps);
    for (int c = 0; c < 3; c++) {
      vbar[c * nidx + k] = ps.vbar[c];
      Pnew[c * nidx + k] = ps.Pnew[c];
    }
    inner_counts[k] = ps.iters;
    if (!conv) fail |= 1;
  }
  tlev_free(&tl);
  eval_free(&e);
  return fail ? ORC_EINNER : ORC_OK;
}
