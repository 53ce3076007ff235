// pic_api.cu -- the C ABI of include/pic.h: context lifetime, set-up
// (Sec. 4.5 projection and the initial Gauss/Lorenz constraints of Sec. 2.3),
// one map evaluation H(j), and the implicit step of Algorithm 1 with the
// type-II Anderson update of Eq. anderson-type-two-update, backtracking and
// the mixed absolute-relative tests of Eq. mixed-nonlinear-tests.
//
// Every vector operation runs in the kernels of field.cu, particle.cu,
// reduce.cu and fft.cu; the host only makes the scalar decisions of the
// outer iteration (accept / backtrack / restart) and solves the <= 8 x 8
// regularised Gram system of the Anderson update.
#include "pic_internal.cuh"
#include "trace.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

// Gauss-Legendre nodes/weights on [0, 1] (Newton on the Legendre recurrence).
void gauss_legendre01(int n, double *t, double *w) {
  for (int i = 0; i < n; i++) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 200; it++) {
      double pk = 1.0, pkm1 = 0.0;
      for (int k = 1; k <= n; k++) {
        double pkm2 = pkm1;
        pkm1 = pk;
        pk = ((2.0 * k - 1.0) * z * pkm1 - (k - 1.0) * pkm2) / k;
      }
      double dp = n * (z * pk - pkm1) / (z * z - 1.0);
      double dz = pk / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) {
        // refresh the derivative at the converged root for the weight
        pk = 1.0; pkm1 = 0.0;
        for (int k = 1; k <= n; k++) {
          double pkm2 = pkm1;
          pkm1 = pk;
          pk = ((2.0 * k - 1.0) * z * pkm1 - (k - 1.0) * pkm2) / k;
        }
        dp = n * (z * pk - pkm1) / (z * z - 1.0);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
        break;
      }
      w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    t[i] = 0.5 * (1.0 - z);
  }
}

namespace {

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
int ilog2(int n) { int l = 0; while ((1 << l) < n) l++; return l; }

void free_all(pic_ctx *ctx) {
  tangent_free(ctx);
  det_free(ctx);
  control_free(ctx);
  void *ptrs[] = {ctx->cell, ctx->off, ctx->P, ctx->w, ctx->sp, ctx->id, ctx->Am, ctx->v0,
                  ctx->vbar, ctx->Pnew, ctx->iters, ctx->u_in, ctx->tmp_d, ctx->tmp_i, ctx->psum,
                  ctx->phi_h, ctx->psi_h, ctx->rho_h, ctx->A_h, ctx->U_h, ctx->A_real, ctx->J_acc,
                  ctx->phi1_h, ctx->psi1_h, ctx->rho1_h, ctx->A1_h, ctx->U1_h, ctx->jh,
                  ctx->work_h, ctx->A1_real, ctx->scr_r, ctx->nodes, ctx->nodes_u, ctx->Jorb,
                  ctx->Jorb_h, ctx->H, ctx->j, ctx->r, ctx->jt, ctx->Ht, ctx->rt, ctx->dir,
                  ctx->dJ, ctx->dR, ctx->tw[0], ctx->tw[1], ctx->tw[2], ctx->red, ctx->cnt_dev,
                  ctx->A_real_f, ctx->cnt_sort, ctx->keys, ctx->tmp_l, ctx->nodes_f,
                  ctx->nodes_u_f, ctx->rep_dev, ctx->dep_rec};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (ctx->red_host) cudaFreeHost(ctx->red_host);
  if (ctx->psum_host) cudaFreeHost(ctx->psum_host);
  if (ctx->cnt_host) cudaFreeHost(ctx->cnt_host);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
}

int alloc_mesh(pic_ctx *ctx) {
  const size_t Ng = ctx->g.Ng, d = ctx->g.dim;
  const size_t C = sizeof(double2), R = sizeof(double);
  double2 **cbufs1[] = {&ctx->phi_h, &ctx->psi_h, &ctx->rho_h, &ctx->phi1_h, &ctx->psi1_h,
                        &ctx->rho1_h};
  for (double2 **b : cbufs1) CK(cudaMalloc((void **)b, C * Ng));
  double2 **cbufs3[] = {&ctx->A_h, &ctx->U_h, &ctx->A1_h, &ctx->U1_h, &ctx->jh, &ctx->Jorb_h};
  for (double2 **b : cbufs3) CK(cudaMalloc((void **)b, C * 3 * Ng));
  CK(cudaMalloc((void **)&ctx->work_h, C * (d + 6) * Ng));
  double **rbufs3[] = {&ctx->A_real, &ctx->J_acc, &ctx->A1_real, &ctx->Jorb, &ctx->H, &ctx->j,
                       &ctx->r, &ctx->jt, &ctx->Ht, &ctx->rt, &ctx->dir};
  for (double **b : rbufs3) CK(cudaMalloc((void **)b, R * 3 * Ng));
  CK(cudaMalloc((void **)&ctx->scr_r, R * 4 * Ng));
  CK(cudaMalloc((void **)&ctx->cnt_sort, sizeof(int32_t) * Ng));
  if (ctx->rsize == 4) CK(cudaMalloc(&ctx->A_real_f, sizeof(float) * 3 * Ng));
  int M = std::max(ctx->opt.anderson_m, 1);
  CK(cudaMalloc((void **)&ctx->dJ, R * 3 * Ng * M));
  CK(cudaMalloc((void **)&ctx->dR, R * 3 * Ng * M));
  CK(cudaMalloc(&ctx->nodes, (size_t)ctx->rsize * node_record_len((int)d) * Ng));
  CK(cudaMalloc(&ctx->nodes_u, (size_t)ctx->rsize * 4 * Ng));
  if (ctx->opt.fp32_first) {
    CK(cudaMalloc((void **)&ctx->nodes_f, sizeof(float) * node_record_len((int)d) * Ng));
    CK(cudaMalloc((void **)&ctx->nodes_u_f, sizeof(float) * 4 * Ng));
  }
  // block partials of the reductions: compensated (sum, error) pairs of up
  // to 3 quantities per block (field.cu), 8 doubles per block (reduce.cu)
  size_t nred = 8 * (Ng / 256 + 2) + 1024 * 48 + 64;
  CK(cudaMalloc((void **)&ctx->red, R * nred));
  CK(cudaMallocHost((void **)&ctx->red_host, R * 64));
  CK(cudaMalloc((void **)&ctx->rep_dev, R * 8));
  CK(cudaMalloc((void **)&ctx->cnt_dev, sizeof(EvalCounters)));
  CK(cudaMallocHost((void **)&ctx->cnt_host, sizeof(EvalCounters)));
  CK(cudaEventCreate(&ctx->ev0));
  CK(cudaEventCreate(&ctx->ev1));
  int e = control_alloc(ctx);
  if (e) return e;
  double2 *zc[] = {ctx->phi_h, ctx->psi_h, ctx->rho_h};
  for (double2 *b : zc) CK(cudaMemsetAsync(b, 0, C * Ng, ctx->st));
  CK(cudaMemsetAsync(ctx->A_h, 0, C * 3 * Ng, ctx->st));
  CK(cudaMemsetAsync(ctx->U_h, 0, C * 3 * Ng, ctx->st));
  CK(cudaMemsetAsync(ctx->A_real, 0, R * 3 * Ng, ctx->st));
  CK(cudaMemsetAsync(ctx->A1_real, 0, R * 3 * Ng, ctx->st));
  CK(cudaMemsetAsync(ctx->J_acc, 0, R * 3 * Ng, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return PIC_OK;
}

}  // namespace

// effective tolerances (reading R9 for the mixed path)
void tolerances(const pic_ctx *ctx, double tol, double *tr, double *ta, double *itr,
                double *ita) {
  double t = tol;
  if (ctx->opt.precision == PIC_MIXED) t = std::max(t, ctx->opt.mixed_tol_floor);
  *tr = t;
  *ta = t * ctx->opt.tol_abs_ratio;
  double ti = tol * ctx->opt.inner_tol_scale;
  if (ctx->opt.precision == PIC_MIXED) ti = std::max(ti, ctx->opt.mixed_tol_floor);
  *itr = ti;
  *ita = ti * ctx->opt.tol_abs_ratio;
}

StepConst make_sc(const pic_ctx *ctx, double itr, double ita) {
  StepConst sc;
  std::memset(&sc, 0, sizeof sc);
  sc.dt = ctx->dt;
  sc.kappa = ctx->opt.kappa;
  for (int s = 0; s < PIC_MAX_SPECIES; s++) {
    sc.qs[s] = s < ctx->nspecies ? ctx->qs[s] : 0.0;
    sc.ms[s] = s < ctx->nspecies ? ctx->ms[s] : 1.0;
  }
  sc.tau_r = itr;
  sc.tau_a = ita;
  sc.inner_max = ctx->opt.inner_max;
  sc.ngl = ctx->opt.gl_points > 0 ? ctx->opt.gl_points : ctx->g.dim + 1;
  sc.warm = ctx->opt.inner_warm_start ? 1 : 0;
  sc.order = ctx->opt.order;
  sc.refine_max = ctx->opt.refine_max;
  gauss_legendre01(sc.ngl, sc.gl_t, sc.gl_w);
  return sc;
}

namespace {

struct Eval {
  EvalCounters cnt;
  double work_p, chain;
};

struct Tests {
  double srms, smax, rms_r;
};

// The launch sequence of one map evaluation H(j) = P J_orb(j) (Sec. 4.5):
// project the trial current, continuity + CN in Fourier space, inner particle
// solves, orbit deposit, projection of the deposit, then r = H - j and the
// sums of the outer tests (Eq. mixed-nonlinear-tests).  Nothing here waits
// for the device, so the sequence can be captured into a CUDA graph.
int eval_enqueue(pic_ctx *ctx, const double *jdev, double *Hdev, double *rdev,
                 const StepConst &sc, int final_pass, double tr, double ta) {
  int e;
  if ((e = field_evaluate(ctx, jdev, final_pass))) return e;
  if ((e = particles_map_launch(ctx, sc, final_pass))) return e;
  // H = P J_orb with the real-space form of the Nyquist projector
  if ((e = field_project_real(ctx, ctx->Jorb, Hdev, 3))) return e;
  if ((e = resid_launch(ctx, Hdev, jdev, rdev, tr, ta))) return e;
  return PIC_OK;
}

}  // namespace

void graphs_clear(pic_ctx *ctx) {
  for (int k = 0; k < ctx->ngraphs; k++) cudaGraphExecDestroy(ctx->graphs[k].exec);
  ctx->ngraphs = 0;
  control_graphs_clear(ctx);
}

namespace {

// Queue one evaluation: replay its captured graph when this buffer set,
// pass kind and tolerance were seen before, otherwise capture it (falling back
// to direct launches if the stream cannot be captured).
int eval_launch(pic_ctx *ctx, const double *jdev, double *Hdev, double *rdev,
                const StepConst &sc, int final_pass, double tr, double ta) {
  ctx->map_final = final_pass;
  if (ctx->graphs_off || ctx->np == 0)
    return eval_enqueue(ctx, jdev, Hdev, rdev, sc, final_pass, tr, ta);
  for (int k = 0; k < ctx->ngraphs; k++) {
    const pic_ctx::GraphEntry &g = ctx->graphs[k];
    if (g.j == jdev && g.H == Hdev && g.r == rdev && g.phi == ctx->phi_h && g.A == ctx->A_real &&
        g.final_pass == final_pass && g.tr == tr && g.ta == ta && g.itr == sc.tau_r &&
        g.ita == sc.tau_a && g.np == ctx->np) {
      CK(cudaGraphLaunch(g.exec, ctx->st));
      ctx->launches += g.nkern;
      return PIC_OK;
    }
  }
  if (ctx->ngraphs == 16) graphs_clear(ctx);
  long long before = ctx->launches;
  if (cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    ctx->graphs_off = 1;
    return eval_enqueue(ctx, jdev, Hdev, rdev, sc, final_pass, tr, ta);
  }
  int e = eval_enqueue(ctx, jdev, Hdev, rdev, sc, final_pass, tr, ta);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(ctx->st, &graph);
  if (e || ce != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    ctx->graphs_off = 1;
    ctx->launches = before;
    if (e && e != PIC_ECUDA) return e;
    return eval_enqueue(ctx, jdev, Hdev, rdev, sc, final_pass, tr, ta);
  }
  cudaGraphExec_t exec = nullptr;
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    ctx->graphs_off = 1;
    ctx->launches = before;
    return eval_enqueue(ctx, jdev, Hdev, rdev, sc, final_pass, tr, ta);
  }
  pic_ctx::GraphEntry &g = ctx->graphs[ctx->ngraphs++];
  g.j = jdev; g.H = Hdev; g.r = rdev; g.phi = ctx->phi_h; g.A = ctx->A_real;
  g.final_pass = final_pass; g.tr = tr; g.ta = ta; g.itr = sc.tau_r; g.ita = sc.tau_a;
  g.np = ctx->np;
  g.nkern = (int)(ctx->launches - before);
  g.exec = exec;
  CK(cudaGraphLaunch(exec, ctx->st));
  return PIC_OK;
}

// One evaluation: queue it, wait once, read the counters and the test sums.
int eval_map(pic_ctx *ctx, const double *jdev, double *Hdev, double *rdev, const StepConst &sc,
             int final_pass, double tr, double ta, Eval *ev, Tests *t) {
  TraceRange trace(final_pass ? "map_eval_verify" : "map_eval");
  int e;
  if ((e = eval_launch(ctx, jdev, Hdev, rdev, sc, final_pass, tr, ta))) return e;
  CK(cudaStreamSynchronize(ctx->st));
  if ((e = particles_map_finish(ctx, &ev->work_p, &ev->chain, &ev->cnt))) return e;
  if (ev->cnt.status) {
    ctx->err = (ev->cnt.status & PIC_ST_WAIT)
                   ? "a bounded device wait gave up (status bits " +
                         std::to_string(ev->cnt.status) + ")"
                   : "inner particle solve failed (status bits " + std::to_string(ev->cnt.status) +
                         ")";
    return PIC_EINNER;
  }
  ResidSums s;
  resid_finish(ctx, &s);
  double n3 = 3.0 * ctx->g.Ng;
  t->rms_r = std::sqrt(s.r2 / n3);
  t->srms = t->rms_r / (ta + 0.5 * tr * (std::sqrt(s.H2 / n3) + std::sqrt(s.j2 / n3)));
  t->smax = s.smax;
  return PIC_OK;
}

// Gaussian elimination with partial pivoting; false if singular / not finite
bool solve_small(int m, double *A, double *b) {
  for (int c = 0; c < m; c++) {
    int piv = c;
    for (int r = c + 1; r < m; r++)
      if (std::fabs(A[r * m + c]) > std::fabs(A[piv * m + c])) piv = r;
    if (A[piv * m + c] == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < m; k++) std::swap(A[c * m + k], A[piv * m + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < m; r++) {
      double f = A[r * m + c] / A[c * m + c];
      for (int k = c; k < m; k++) A[r * m + k] -= f * A[c * m + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = m - 1; c >= 0; c--) {
    double s = b[c];
    for (int k = c + 1; k < m; k++) s -= A[c * m + k] * b[k];
    b[c] = s / A[c * m + c];
    if (!std::isfinite(b[c])) return false;
  }
  return true;
}

// Inexact Newton-Krylov outer iteration (option nonlinear_solver): Algorithm
// 1's tests, backtracking and verifying evaluation, with the Newton direction
// (I - H'(j)) d = r of nk_direction in place of the Anderson / damped Picard
// directions.  The caller has evaluated H at the first iterate (j, H, r, T).
int newton_krylov_outer(pic_ctx *ctx, const StepConst &sc, double tr, double ta, pic_report &R,
                        Eval &ev, Tests &T, double *&j, double *&H, double *&r, double *&jt,
                        double *&Ht, double *&rt, bool &done) {
  NkState *nk = nullptr;
  struct Release {
    NkState **p;
    ~Release() { nk_end(*p); }
  } release{&nk};
  int e = nk_begin(ctx, sc, &nk);
  if (e) return e;
  const size_t N3 = (size_t)3 * ctx->g.Ng;
  int status = PIC_OK;
  double rms_prev = 0.0, eta_prev = 0.1;
  for (int k = 0; k < ctx->opt.outer_max; k++) {
    TraceRange trace_k("outer_iteration");
    R.outer_iters = k + 1;
    R.res_scaled_rms = T.srms;
    R.res_scaled_max = T.smax;
    if (T.srms <= 1.0 && T.smax <= 1.0) {
      status = eval_map(ctx, j, H, r, sc, 1, tr, ta, &ev, &T);
      R.map_evals++;
      if (status != PIC_OK) return status;
      R.res_scaled_rms = T.srms;
      R.res_scaled_max = T.smax;
      if (!(T.srms <= 1.0 && T.smax <= 1.0)) {
        ctx->err = "verification evaluation failed the outer tests";
        return PIC_EOUTER;
      }
      done = true;
      return PIC_OK;
    }
    // forcing term: Eisenstat-Walker choice 2 (gamma 0.9, exponent 2) with
    // its safeguard, at most 0.5, and no smaller than the reduction that
    // still brings the scaled residual to half the test's bound
    double eta = 0.1;
    if (k > 0) {
      const double q = T.rms_r / rms_prev;
      eta = 0.9 * q * q;
      if (0.9 * eta_prev * eta_prev > 0.1) eta = std::fmax(eta, 0.9 * eta_prev * eta_prev);
    }
    eta = std::fmin(std::fmax(eta, 0.5 / T.srms), 0.5);
    int its = 0;
    e = nk_direction(ctx, nk, r, eta, ctx->dir, &its);
    R.jvp_evals += its;
    if (e) return e;
    bool accepted = false;
    Tests Tt = T;
    double alpha = 1.0;
    for (int lvl = 0; lvl < ctx->opt.backtrack_levels; lvl++, alpha *= 0.5) {
      if ((e = lincomb(ctx, jt, j, 1.0, ctx->dir, alpha, N3))) return e;
      status = eval_map(ctx, jt, Ht, rt, sc, 0, tr, ta, &ev, &Tt);
      R.map_evals++;
      if (status != PIC_OK) return status;
      if (Tt.srms <= (1.0 - ctx->opt.decrease_coef * alpha) * T.srms &&
          Tt.smax <= ctx->opt.growth_limit * T.smax) {
        accepted = true;
        break;
      }
    }
    if (!accepted) {
      ctx->err = "no accepted Newton step";
      return PIC_EOUTER;
    }
    rms_prev = T.rms_r;
    eta_prev = eta;
    std::swap(j, jt);
    std::swap(H, Ht);
    std::swap(r, rt);
    T = Tt;
  }
  ctx->err = "outer iteration limit reached";
  return PIC_EOUTER;
}

int finish_report(pic_ctx *ctx, pic_report *R) {
  int e;
  double K, W, gr, lr;
  if ((e = particles_kinetic(ctx, &K))) return e;
  if ((e = field_energy(ctx, ctx->phi_h, ctx->A_h, ctx->U_h, &W))) return e;
  if ((e = field_constraints(ctx, &gr, &lr))) return e;
  R->K = K;
  R->W = W;
  R->E_tot = K + W;
  R->gauss_rms = gr;
  R->lorenz_rms = lr;
  R->rel_dE = ctx->E0 != 0.0 ? (R->E_tot - ctx->E0) / ctx->E0 : 0.0;
  return PIC_OK;
}

int set_fields_real(pic_ctx *ctx, const double *src_dev, double2 *dst, int ncomp) {
  int e;
  if ((e = field_real_to_complex(ctx, src_dev, dst, ncomp))) return e;
  return fft_nd(ctx, dst, ncomp, -1);
}

int get_field_real(pic_ctx *ctx, const double2 *src, int ncomp, double *out, int on_device) {
  const int Ng = ctx->g.Ng;
  for (int c = 0; c < ncomp; c++) {
    CK(cudaMemcpyAsync(ctx->work_h, src + (size_t)c * Ng, sizeof(double2) * Ng,
                       cudaMemcpyDeviceToDevice, ctx->st));
    int e = fft_nd(ctx, ctx->work_h, 1, +1);
    if (e) return e;
    double *dst = on_device ? out + (size_t)c * Ng : ctx->scr_r;
    if ((e = field_complex_to_real(ctx, ctx->work_h, dst, 1, 1.0 / Ng))) return e;
    if (!on_device)
      CK(cudaMemcpyAsync(out + (size_t)c * Ng, ctx->scr_r, sizeof(double) * Ng,
                         cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  return PIC_OK;
}

int copy_in(pic_ctx *ctx, double *dst_dev, const double *src, size_t n, int on_device) {
  CK(cudaMemcpyAsync(dst_dev, src, sizeof(double) * n,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->st));
  return PIC_OK;
}

}  // namespace

namespace {

int set_particles(pic_ctx *ctx, int64_t n, const int32_t *species, const int32_t *cell,
                  const double *x, const double *u_or_P, int is_canonical, const double *w,
                  int on_device) {
  tangent_free(ctx);  // its arrays follow the particle storage
  if (!ctx) return PIC_EARG;
  if (n < 0 || (n > 0 && (!x || !u_or_P || !w))) {
    ctx->err = "pic_set_particles: bad arguments";
    return PIC_EARG;
  }
  if (species && !on_device)
    for (int64_t i = 0; i < n; i++)
      if (species[i] < 0 || species[i] >= ctx->nspecies) {
        ctx->err = "pic_set_particles: species index out of range";
        return PIC_EARG;
      }
  if (cell && !on_device)
    for (int l = 0; l < ctx->g.dim; l++)
      for (int64_t i = 0; i < n; i++)
        if (cell[l * n + i] < 0 || cell[l * n + i] >= ctx->g.n[l] ||
            !(x[l * n + i] >= -0.5 && x[l * n + i] < 0.5)) {
          ctx->err = "pic_set_particles_local: node index or offset out of range";
          return PIC_EARG;
        }
  graphs_clear(ctx);
  ctx->started = 0;
  int e = particles_alloc(ctx, n);
  if (e) return e;
  ctx->np = n;
  if ((e = particles_load(ctx, species, cell, x, u_or_P, is_canonical, w, on_device))) {
    // a refused load leaves an empty, unstarted context
    ctx->np = 0;
    ctx->have_particles = 0;
    return e;
  }
  ctx->pending_mech = !is_canonical;
  ctx->have_particles = 1;
  return PIC_OK;
}

}  // namespace

extern "C" {

void pic_default_options(pic_options *o) {
  std::memset(o, 0, sizeof *o);
  o->kappa = 1.0;
  o->sigma1 = 1.0;
  o->sigma2 = 1.0;
  o->rho_bg = 0.0;
  o->project_nyquist = 1;
  o->gl_points = 0;
  o->inner_max = 64;
  o->outer_max = 80;
  o->anderson_m = 4;
  o->anderson_start = 2;
  o->backtrack_levels = 7;
  o->beta = 0.5;
  o->lambda = 1e-12;
  o->decrease_coef = 1e-4;
  o->growth_limit = 1.2;
  o->tol_abs_ratio = 0.01;
  o->inner_tol_scale = 1.0;
  o->precision = PIC_FP64;
  o->mixed_tol_floor = 1e-5;
  o->sort_every = 10;
  o->cuda_stream = nullptr;
  o->inner_warm_start = 0;
  o->order = 2;
  o->refine_max = 0;
  o->deterministic_deposit = 0;
}

int pic_init(pic_ctx **out, const pic_grid *grid, const pic_species *species, int nspecies,
             double dt, const pic_options *opt) {
  if (!out) return PIC_EARG;
  *out = nullptr;
  if (!grid || !species || nspecies < 1 || nspecies > PIC_MAX_SPECIES || !(dt > 0.0))
    return PIC_EARG;
  if (grid->dim < 1 || grid->dim > 3) return PIC_EARG;
  for (int a = 0; a < grid->dim; a++)
    if (!is_pow2(grid->n[a]) || grid->n[a] < 4 || grid->n[a] > 4096 || !(grid->L[a] > 0.0))
      return PIC_EARG;
  for (int s = 0; s < nspecies; s++)
    if (!(species[s].m > 0.0)) return PIC_EARG;
  pic_options o;
  if (opt) o = *opt;
  else pic_default_options(&o);
  if (o.gl_points < 0 || o.gl_points > PIC_MAX_GL || o.inner_max < 1 || o.outer_max < 1 ||
      o.anderson_m < 0 || o.anderson_m > PIC_MAX_ANDERSON || o.backtrack_levels < 1 ||
      (o.precision != PIC_FP64 && o.precision != PIC_MIXED) || !(o.kappa > 0.0) ||
      !(o.sigma1 > 0.0) || !(o.sigma2 > 0.0) || (o.order != 1 && o.order != 2) ||
      o.refine_max < 0 || o.refine_max > 3 ||
      (o.deterministic_deposit && (o.precision != PIC_FP64 || o.refine_max != 0)) ||
      (o.nonlinear_solver != PIC_SOLVER_ANDERSON &&
       o.nonlinear_solver != PIC_SOLVER_NEWTON_KRYLOV) ||
      (o.nonlinear_solver == PIC_SOLVER_NEWTON_KRYLOV &&
       (o.precision != PIC_FP64 || o.order != 2 || o.refine_max != 0 || o.inner_warm_start ||
        o.deterministic_deposit)) ||
      (o.fp32_first && (o.precision != PIC_FP64 || o.order != 2 || o.refine_max != 0 ||
                        o.nonlinear_solver != PIC_SOLVER_ANDERSON || o.host_control ||
                        o.deterministic_deposit)))
    return PIC_EARG;
  // the deterministic deposit's node gather spans at least 5 nodes per dimension
  if (o.deterministic_deposit)
    for (int a = 0; a < grid->dim; a++)
      if (grid->n[a] < 8) return PIC_EARG;
  pic_ctx *ctx = new (std::nothrow) pic_ctx();
  if (!ctx) return PIC_ENOMEM;
  ctx->opt = o;
  ctx->st = (cudaStream_t)o.cuda_stream;
  if (!ctx->st) {
    // the legacy default stream cannot be captured into graphs: use a
    // blocking stream of our own, which orders itself with the legacy stream
    if (cudaStreamCreate(&ctx->own_st) != cudaSuccess) {
      delete ctx;
      return PIC_ECUDA;
    }
    ctx->st = ctx->own_st;
  }
  ctx->dt = dt;
  ctx->nspecies = nspecies;
  for (int s = 0; s < nspecies; s++) {
    ctx->qs[s] = species[s].q;
    ctx->ms[s] = species[s].m;
  }
  Geom &g = ctx->g;
  g.dim = grid->dim;
  g.Ng = 1;
  g.dV = 1.0;
  for (int a = 0; a < 3; a++) {
    bool act = a < g.dim;
    g.n[a] = act ? grid->n[a] : 1;
    g.logn[a] = act ? ilog2(g.n[a]) : 0;
    g.L[a] = act ? grid->L[a] : 1.0;
    g.x0[a] = act ? grid->x0[a] : 0.0;
    g.dx[a] = g.L[a] / g.n[a];
    g.Ng *= g.n[a];
    if (act) g.dV *= g.dx[a];
  }
  ctx->rsize = o.precision == PIC_MIXED ? 4 : 8;
  int e = alloc_mesh(ctx);
  if (!e) e = fft_init(ctx);
  if (!e) e = particles_alloc(ctx, 1);
  if (e) {
    free_all(ctx);
    if (ctx->own_st) cudaStreamDestroy(ctx->own_st);
    delete ctx;
    return e == PIC_ECUDA ? PIC_ENOMEM : e;
  }
  *out = ctx;
  return PIC_OK;
}

void pic_free(pic_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->st);
  graphs_clear(ctx);
  free_all(ctx);
  if (ctx->own_st) cudaStreamDestroy(ctx->own_st);
  delete ctx;
}

const char *pic_last_error(const pic_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int pic_get_stats(const pic_ctx *ctx, pic_stats *out) {
  if (!ctx || !out) return PIC_EARG;
  out->launches = ctx->launches;
  out->map_launches = ctx->map_launches;
  out->map_ms = ctx->map_ms;
  out->pushes = ctx->pushes;
  out->inner_iters = ctx->inner_iters;
  out->pieces = ctx->pieces;
  out->refined = ctx->refined;
  return PIC_OK;
}

int pic_reset_stats(pic_ctx *ctx) {
  if (!ctx) return PIC_EARG;
  ctx->launches = ctx->map_launches = ctx->pushes = ctx->inner_iters = ctx->pieces = 0;
  ctx->refined = 0;
  ctx->map_ms = 0.0;
  return PIC_OK;
}

int64_t pic_num_particles(const pic_ctx *ctx) { return ctx ? ctx->np : -1; }

int pic_set_particles(pic_ctx *ctx, int64_t n, const int32_t *species, const double *x,
                      const double *u_or_P, int is_canonical, const double *w, int on_device) {
  if (!ctx) return PIC_EARG;
  return set_particles(ctx, n, species, nullptr, x, u_or_P, is_canonical, w, on_device);
}

int pic_set_particles_local(pic_ctx *ctx, int64_t n, const int32_t *species, const int32_t *cell,
                            const double *offset, const double *u_or_P, int is_canonical,
                            const double *w, int on_device) {
  if (!ctx) return PIC_EARG;
  if (n > 0 && !cell) {
    ctx->err = "pic_set_particles_local: bad arguments";
    return PIC_EARG;
  }
  return set_particles(ctx, n, species, cell, offset, u_or_P, is_canonical, w, on_device);
}

int pic_set_potentials(pic_ctx *ctx, const double *A, const double *U, int on_device) {
  if (!ctx) return PIC_EARG;
  size_t N3 = (size_t)3 * ctx->g.Ng;
  if (A) { int e = copy_in(ctx, ctx->A_real, A, N3, on_device); if (e) return e; }
  else CK(cudaMemsetAsync(ctx->A_real, 0, sizeof(double) * N3, ctx->st));
  // U is staged in A1_real until pic_start transforms it
  if (U) { int e = copy_in(ctx, ctx->A1_real, U, N3, on_device); if (e) return e; }
  else CK(cudaMemsetAsync(ctx->A1_real, 0, sizeof(double) * N3, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->started = 0;
  return PIC_OK;
}

int pic_start(pic_ctx *ctx, pic_report *out) {
  if (!ctx) return PIC_EARG;
  TraceRange trace("pic_start");
  tangent_free(ctx);
  const int Ng = ctx->g.Ng;
  int e;
  // project A and U (Sec. 4.5) and bring A back to real space
  if ((e = set_fields_real(ctx, ctx->A_real, ctx->A_h, 3))) return e;
  if ((e = field_project_h(ctx, ctx->A_h, 3))) return e;
  if ((e = set_fields_real(ctx, ctx->A1_real, ctx->U_h, 3))) return e;
  if ((e = field_project_h(ctx, ctx->U_h, 3))) return e;
  CK(cudaMemcpyAsync(ctx->work_h, ctx->A_h, sizeof(double2) * 3 * Ng, cudaMemcpyDeviceToDevice,
                     ctx->st));
  if ((e = fft_nd(ctx, ctx->work_h, 3, +1))) return e;
  if ((e = field_complex_to_real(ctx, ctx->work_h, ctx->A_real, 3, 1.0 / Ng))) return e;
  if ((e = particles_refresh_A(ctx))) return e;
  if (ctx->pending_mech) {
    if ((e = particles_form_P(ctx))) return e;
    ctx->pending_mech = 0;
  }
  // point deposits of rho^0 and J^0 (readings R10, R11), projected
  double *rho = ctx->scr_r;
  std::vector<double> bg(Ng, ctx->opt.rho_bg);
  CK(cudaMemcpyAsync(rho, bg.data(), sizeof(double) * Ng, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemsetAsync(ctx->J_acc, 0, sizeof(double) * 3 * Ng, ctx->st));
  if ((e = det_alloc(ctx))) return e;
  if (ctx->opt.deterministic_deposit) {
    if ((e = det_point_deposit(ctx, rho, ctx->J_acc, make_sc(ctx, 0.0, 0.0)))) return e;
  } else if ((e = particles_point_deposit(ctx, rho, ctx->J_acc))) {
    return e;
  }
  if ((e = set_fields_real(ctx, rho, ctx->rho_h, 1))) return e;
  if ((e = field_project_h(ctx, ctx->rho_h, 1))) return e;
  if ((e = set_fields_real(ctx, ctx->J_acc, ctx->jh, 3))) return e;
  if ((e = field_project_h(ctx, ctx->jh, 3))) return e;
  CK(cudaMemcpyAsync(ctx->work_h, ctx->jh, sizeof(double2) * 3 * Ng, cudaMemcpyDeviceToDevice,
                     ctx->st));
  if ((e = fft_nd(ctx, ctx->work_h, 3, +1))) return e;
  if ((e = field_complex_to_real(ctx, ctx->work_h, ctx->J_acc, 3, 1.0 / Ng))) return e;
  if ((e = field_initial_constraints(ctx))) return e;
  CK(cudaStreamSynchronize(ctx->st));
  pic_report R;
  std::memset(&R, 0, sizeof R);
  ctx->E0 = 0.0;
  if ((e = finish_report(ctx, &R))) return e;
  ctx->E0 = R.E_tot;
  R.rel_dE = 0.0;
  if (ctx->opt.sort_every > 0 && (e = particles_sort(ctx))) return e;
  ctx->started = 1;
  ctx->steps_done = 0;
  if (out) *out = R;
  return PIC_OK;
}

int pic_eval_map(pic_ctx *ctx, const double *j, double tol, double *H, double *vbar,
                 double *Pnew, int32_t *inner_counts, int on_device) {
  if (!ctx) return PIC_EARG;
  if (!ctx->started) {
    ctx->err = "pic_eval_map before pic_start";
    return PIC_ESTATE;
  }
  const size_t N3 = (size_t)3 * ctx->g.Ng;
  double tr, ta, itr, ita;
  tolerances(ctx, tol, &tr, &ta, &itr, &ita);
  StepConst sc = make_sc(ctx, itr, ita);
  int e;
  if ((e = particles_step_start(ctx))) return e;
  if (j) { if ((e = copy_in(ctx, ctx->jt, j, N3, on_device))) return e; }
  else CK(cudaMemcpyAsync(ctx->jt, ctx->J_acc, sizeof(double) * N3, cudaMemcpyDeviceToDevice,
                          ctx->st));
  Eval ev;
  Tests T;
  int st = eval_map(ctx, ctx->jt, ctx->Ht, ctx->rt, sc, 0, tr, ta, &ev, &T);
  if (st != PIC_OK && st != PIC_EINNER) return st;
  if (H && st == PIC_OK)
    CK(cudaMemcpyAsync(H, ctx->Ht, sizeof(double) * N3,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->st));
  if ((e = particles_export_eval(ctx, vbar, Pnew, inner_counts, on_device))) return e;
  CK(cudaStreamSynchronize(ctx->st));
  return st;
}

int pic_step(pic_ctx *ctx, double tol, pic_report *out) {
  if (!ctx) return PIC_EARG;
  TraceRange trace("pic_step");
  pic_report R;
  std::memset(&R, 0, sizeof R);
  if (!ctx->started) {
    ctx->err = "pic_step before pic_start";
    R.status = PIC_ESTATE;
    if (out) *out = R;
    return PIC_ESTATE;
  }
  const size_t N3 = (size_t)3 * ctx->g.Ng;
  double tr, ta, itr, ita;
  tolerances(ctx, tol, &tr, &ta, &itr, &ita);
  StepConst sc = make_sc(ctx, itr, ita);
  const int M = ctx->opt.anderson_m;
  int e;
  if ((e = particles_step_start(ctx))) return e;
  double *j = ctx->j, *H = ctx->H, *r = ctx->r, *jt = ctx->jt, *Ht = ctx->Ht, *rt = ctx->rt;
  Eval ev;
  Tests T;
  int status = PIC_OK;
  bool done = false;
  int ran = 0;
  const bool newton = ctx->opt.nonlinear_solver == PIC_SOLVER_NEWTON_KRYLOV;
  if (!ctx->opt.host_control && !newton) {
    // the whole outer iteration on the device (control.cu)
    StepOutcome so;
    int from_j = 0, evals0 = 0, iters0 = 0;
    if (ctx->opt.fp32_first) {
      // FP32 stage: FP32 arithmetic on the FP64 particle state down to the
      // FP32 floor of the tolerance, no verification; the FP64 iteration
      // then continues from its last accepted current (fresh Anderson
      // history: the map has changed)
      const double t32 = std::max(tol, ctx->opt.mixed_tol_floor);
      double tr32, ta32, itr32, ita32;
      tolerances(ctx, t32, &tr32, &ta32, &itr32, &ita32);
      ctx->eval_f32 = 1;
      int ran32 = 0;
      e = step_control_device(ctx, make_sc(ctx, itr32, ita32), tr32, ta32, &so, &ran32, 0, 0);
      ctx->eval_f32 = 0;
      if (e) return e;
      if (ran32) {
        from_j = 1;  // even a failed FP32 stage leaves an accepted iterate in j
        evals0 = so.map_evals;
        iters0 = so.outer_iters;
        R.fp32_evals = so.map_evals;
      }
    }
    if ((e = step_control_device(ctx, sc, tr, ta, &so, &ran, from_j, 1))) return e;
    if (ran) {
      status = so.status;
      done = status == PIC_OK;
      R.outer_iters = iters0 + so.outer_iters;
      R.map_evals = evals0 + so.map_evals;
      R.res_scaled_rms = so.res_srms;
      R.res_scaled_max = so.res_smax;
      ev.work_p = so.work_p;
      ev.chain = so.chain;
      std::memset(&ev.cnt, 0, sizeof ev.cnt);
      ev.cnt.inner_max = so.inner_max;
      ev.cnt.inner_sum = so.inner_sum;
      ev.cnt.refined = so.refined;
      if (status == PIC_EINNER) ctx->err = "inner particle solve failed";
      else if (status == PIC_EOUTER)
        ctx->err = so.why == 4 ? "verification evaluation failed the outer tests"
                   : so.why == 3 ? "no accepted outer direction"
                                 : "outer iteration limit reached";
    }
  }
  if (!ran) {
  CK(cudaMemcpyAsync(j, ctx->J_acc, sizeof(double) * N3, cudaMemcpyDeviceToDevice, ctx->st));
  status = eval_map(ctx, j, H, r, sc, 0, tr, ta, &ev, &T);
  R.map_evals = 1;
  if (status != PIC_OK && status != PIC_EINNER) return status;
  if (newton && status == PIC_OK) {
    status = newton_krylov_outer(ctx, sc, tr, ta, R, ev, T, j, H, r, jt, Ht, rt, done);
    if (status != PIC_OK && status != PIC_EINNER && status != PIC_EOUTER) return status;
  }
  if (!newton) {
  // Anderson history: ring of M columns, oldest at hist0
  int mh = 0, hist0 = 0;
  for (int k = 0; status == PIC_OK && k < ctx->opt.outer_max; k++) {
    TraceRange trace_k("outer_iteration");
    R.outer_iters = k + 1;
    R.res_scaled_rms = T.srms;
    R.res_scaled_max = T.smax;
    if (T.srms <= 1.0 && T.smax <= 1.0) {
      // verify by re-evaluating the map at the candidate current
      status = eval_map(ctx, j, H, r, sc, 1, tr, ta, &ev, &T);
      R.map_evals++;
      if (status != PIC_OK) break;
      R.res_scaled_rms = T.srms;
      R.res_scaled_max = T.smax;
      if (!(T.srms <= 1.0 && T.smax <= 1.0)) {
        status = PIC_EOUTER;
        ctx->err = "verification evaluation failed the outer tests";
        break;
      }
      done = true;
      break;
    }
    bool have_anderson = false;
    if (k + 1 >= ctx->opt.anderson_start && mh > 0) {  // iterations counted from 1
      const double *cols[PIC_MAX_ANDERSON], *jcols[PIC_MAX_ANDERSON];
      for (int c = 0; c < mh; c++) {
        int slot = (hist0 + c) % M;
        cols[c] = ctx->dR + (size_t)slot * N3;
        jcols[c] = ctx->dJ + (size_t)slot * N3;
      }
      const double *a[48], *b[48];
      int np = 0;
      for (int p = 0; p < mh; p++)
        for (int q = p; q < mh; q++) { a[np] = cols[p]; b[np] = cols[q]; np++; }
      for (int p = 0; p < mh; p++) { a[np] = cols[p]; b[np] = r; np++; }
      double dv[48];
      if ((e = dots(ctx, a, b, np, dv))) return e;
      double G[PIC_MAX_ANDERSON * PIC_MAX_ANDERSON], gam[PIC_MAX_ANDERSON], tr_g = 0.0;
      int idx = 0;
      for (int p = 0; p < mh; p++)
        for (int q = p; q < mh; q++) { G[p * mh + q] = G[q * mh + p] = dv[idx++]; }
      for (int p = 0; p < mh; p++) { gam[p] = dv[idx++]; tr_g += G[p * mh + p]; }
      for (int p = 0; p < mh; p++) G[p * mh + p] += ctx->opt.lambda * tr_g / mh;
      if (std::isfinite(tr_g) && tr_g > 0.0 && solve_small(mh, G, gam)) {
        have_anderson = true;
        if ((e = axpy_dir(ctx, ctx->dir, r, ctx->opt.beta, jcols, cols, gam, mh, N3))) return e;
      } else {
        mh = 0;  // unusable history
      }
    }
    bool accepted = false;
    Tests Tt = T;
    for (int attempt = have_anderson ? 0 : 1; attempt < 2 && !accepted; attempt++) {
      if (attempt == 1 && (e = lincomb(ctx, ctx->dir, r, ctx->opt.beta, r, 0.0, N3))) return e;
      double alpha = 1.0;
      for (int lvl = 0; lvl < ctx->opt.backtrack_levels; lvl++, alpha *= 0.5) {
        if ((e = lincomb(ctx, jt, j, 1.0, ctx->dir, alpha, N3))) return e;
        status = eval_map(ctx, jt, Ht, rt, sc, 0, tr, ta, &ev, &Tt);
        R.map_evals++;
        if (status != PIC_OK) break;
        if (Tt.srms <= (1.0 - ctx->opt.decrease_coef * alpha) * T.srms &&
            Tt.smax <= ctx->opt.growth_limit * T.smax) {
          accepted = true;
          break;
        }
      }
      if (status != PIC_OK) break;
    }
    if (status != PIC_OK) break;
    if (!accepted) {
      status = PIC_EOUTER;
      ctx->err = "no accepted outer direction";
      break;
    }
    if (M > 0) {
      int slot;
      if (mh == M) {
        slot = hist0;
        hist0 = (hist0 + 1) % M;
      } else {
        slot = (hist0 + mh) % M;
        mh++;
      }
      if ((e = diff_into(ctx, ctx->dJ + (size_t)slot * N3, jt, j, N3))) return e;
      if ((e = diff_into(ctx, ctx->dR + (size_t)slot * N3, rt, r, N3))) return e;
      const double grown = ctx->opt.growth_scaled ? Tt.srms / T.srms : Tt.rms_r / T.rms_r;
      if (grown > ctx->opt.growth_limit) { mh = 0; hist0 = 0; }
    }
    std::swap(j, jt);
    std::swap(H, Ht);
    std::swap(r, rt);
    T = Tt;
  }
  if (status == PIC_OK && !done) {
    status = PIC_EOUTER;
    ctx->err = "outer iteration limit reached";
  }
  }  // Anderson
  }  // host-driven outer iteration
  // the forward sensitivity of the converged step (before anything commits)
  if (status == PIC_OK && ctx->tan) {
    status = tangent_solve(ctx, sc, tol);
    if (status != PIC_OK && status != PIC_EOUTER && status != PIC_EINNER) return status;
  }
  // keep the device buffers in their named slots for the next step
  ctx->j = j; ctx->H = H; ctx->r = r; ctx->jt = jt; ctx->Ht = Ht; ctx->rt = rt;
  if (status == PIC_OK) {
    TraceRange trace_c("commit");
    // the commit and every commit-time sum are queued, then read back with
    // one copy and one synchronisation
    if ((e = field_mesh_work_real_queued(ctx, H, ctx->rep_dev))) return e;
    R.chain_rms = ctx->np ? std::sqrt(ev.chain / (3.0 * ctx->np)) : 0.0;
    R.inner_max = ev.cnt.inner_max;
    R.inner_mean = ctx->np ? (double)ev.cnt.inner_sum / ctx->np : 0.0;
    R.refined = (int)ev.cnt.refined;
    if ((e = particles_commit(ctx))) return e;
    if (ctx->tan && (e = tangent_commit(ctx))) return e;
    std::swap(ctx->phi_h, ctx->phi1_h);
    std::swap(ctx->psi_h, ctx->psi1_h);
    std::swap(ctx->rho_h, ctx->rho1_h);
    std::swap(ctx->A_h, ctx->A1_h);
    std::swap(ctx->U_h, ctx->U1_h);
    std::swap(ctx->A_real, ctx->A1_real);
    if ((e = particles_refresh_A(ctx))) return e;
    CK(cudaMemcpyAsync(ctx->J_acc, j, sizeof(double) * N3, cudaMemcpyDeviceToDevice, ctx->st));
    if ((e = particles_kinetic_queued(ctx))) return e;
    if ((e = field_energy_queued(ctx, ctx->rep_dev + 1))) return e;
    if ((e = field_constraints_queued(ctx, ctx->rep_dev + 2))) return e;
    CK(cudaMemcpyAsync(ctx->red_host, ctx->rep_dev, sizeof(double) * 4, cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    const double *rh = ctx->red_host;
    R.work_residual = ctx->dt * (ev.work_p - rh[0] * ctx->g.dV);
    R.K = particles_kinetic_collect(ctx);
    // Parseval for the unnormalised DFT: sum_g |f_g|^2 = sum_k |f_k|^2 / Ng
    R.W = rh[1] * ctx->g.dV / ctx->g.Ng;
    R.E_tot = R.K + R.W;
    R.gauss_rms = std::sqrt(rh[2]) / ctx->g.Ng;
    R.lorenz_rms = std::sqrt(rh[3]) / ctx->g.Ng;
    R.rel_dE = ctx->E0 != 0.0 ? (R.E_tot - ctx->E0) / ctx->E0 : 0.0;
    ctx->steps_done++;
    if (ctx->opt.sort_every > 0 && ctx->steps_done % ctx->opt.sort_every == 0 &&
        (e = particles_sort(ctx)))
      return e;
  }
  R.status = status;
  if (out) *out = R;
  return status;
}

int pic_get_particles(pic_ctx *ctx, double *x, double *P, double *w, int32_t *species,
                      int on_device) {
  if (!ctx) return PIC_EARG;
  return particles_export(ctx, x, P, w, species, on_device);
}

int pic_get_velocities(pic_ctx *ctx, double *u, int on_device) {
  if (!ctx || !u) return PIC_EARG;
  return particles_export_u(ctx, u, on_device);
}

int pic_get_potentials(pic_ctx *ctx, double *phi, double *psi, double *A, double *U, double *rho,
                       double *J, int on_device) {
  if (!ctx) return PIC_EARG;
  int e;
  if (phi && (e = get_field_real(ctx, ctx->phi_h, 1, phi, on_device))) return e;
  if (psi && (e = get_field_real(ctx, ctx->psi_h, 1, psi, on_device))) return e;
  if (rho && (e = get_field_real(ctx, ctx->rho_h, 1, rho, on_device))) return e;
  if (A && (e = get_field_real(ctx, ctx->A_h, 3, A, on_device))) return e;
  if (U && (e = get_field_real(ctx, ctx->U_h, 3, U, on_device))) return e;
  if (J) {
    CK(cudaMemcpyAsync(J, ctx->J_acc, sizeof(double) * 3 * ctx->g.Ng,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  return PIC_OK;
}

int pic_set_state(pic_ctx *ctx, int64_t n, const int32_t *species, const double *x,
                  const double *P, const double *w, const double *phi, const double *psi,
                  const double *A, const double *U, const double *rho, const double *J, double E0,
                  int on_device) {
  if (!ctx) return PIC_EARG;
  if (!phi || !psi || !A || !U || !rho || !J) {
    ctx->err = "pic_set_state: every mesh array is required";
    return PIC_EARG;
  }
  int e = pic_set_particles(ctx, n, species, x, P, 1, w, on_device);
  if (e) return e;
  const size_t Ng = ctx->g.Ng;
  struct {
    const double *src;
    double2 *dst;
    int nc;
  } f[] = {{phi, ctx->phi_h, 1}, {psi, ctx->psi_h, 1}, {rho, ctx->rho_h, 1}, {A, ctx->A_h, 3},
           {U, ctx->U_h, 3}};
  for (auto &it : f) {
    for (int c = 0; c < it.nc; c++) {
      if ((e = copy_in(ctx, ctx->scr_r, it.src + c * Ng, Ng, on_device))) return e;
      if ((e = set_fields_real(ctx, ctx->scr_r, it.dst + c * Ng, 1))) return e;
    }
  }
  if ((e = copy_in(ctx, ctx->A_real, A, 3 * Ng, on_device))) return e;
  if ((e = particles_refresh_A(ctx))) return e;
  if ((e = copy_in(ctx, ctx->J_acc, J, 3 * Ng, on_device))) return e;
  CK(cudaStreamSynchronize(ctx->st));
  if ((e = det_alloc(ctx))) return e;
  ctx->E0 = E0;
  ctx->started = 1;
  ctx->pending_mech = 0;
  return PIC_OK;
}

}  // extern "C"
