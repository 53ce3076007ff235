// tangent.cu -- forward-mode derivatives of the step.  The paper's outer
// solver is the Picard/Anderson iteration of Algorithm 1 and it has no
// tangent; these calls serve Newton-Krylov solvers and gradients:
//  * pic_eval_map_jvp: one evaluation of the outer map H(j) = P J_orb(j)
//    (Sec. 4.5) with its directional derivative dH = H'(j) dj;
//  * pic_tangent_begin / pic_get_tangent / pic_tangent_end: the forward
//    sensitivity of the accepted state, carried through pic_step.  At the
//    converged current j* = H(j*; S) of a step from state S, the tangent dj
//    solves (I - H_j) dj = H_S dS (implicit differentiation of the fixed
//    point), by restarted GMRES on Jacobian-vector products; the tangents of
//    vbar, P^{n+1} and of the CN field step then follow from dj.
//
// The field step is linear in (j, field state) jointly, so its tangent is
// the same CN update applied to the tangents (field_cn_update_into).  The
// particle part is differentiated in forward mode: the particle map of
// map_device.cuh runs on dual numbers (dual.cuh) whose values come from the
// primal gather records and particle state and whose tangents come from the
// tangent records (d grad phi^{1/2}, dA^n, dA^{n+1}) and the particle
// tangents (offset, P, and A^- and v(p^n) derived from them).  The inner
// Picard iteration converges the orbit velocity and its tangent together
// (the tangent of the inner fixed point), the knot-split orbit integrals
// differentiate through their moving piece ends, and the deposit carries
// q (vbar Sbar)' / dV into a second current array.
#include "map_device.cuh"
#include "trace.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace {

constexpr int kKrylov = 20;     // GMRES restart length
constexpr int kRestarts = 6;    // restarts before the tangent solve gives up
// A tangent map evaluation carries the rounding of the deposit's gross
// terms; where the net tangent current is a small part of them (counter-
// streaming beams) GMRES stalls slightly above the requested tolerance.  A
// restart that gains less than a factor two with the relative residual below
// kNoiseFloor ends the solve as converged to the attainable accuracy.
constexpr double kNoiseFloor = 1e-9;

// out[c * so + i] = (a[c * sa + i], b[c * sa + i]) (b may be null: zero tangent)
__global__ void k_zip(const double *__restrict__ a, const double *__restrict__ b,
                      Dual *__restrict__ out, int64_t n, int nc, int64_t sa, int64_t so) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int c = 0; c < nc; c++) out[c * so + i] = Dual(a[c * sa + i], b ? b[c * sa + i] : 0.0);
}

// A_h(x) as a dual number: the value from A^n, the tangent from the moving
// offset (the weights' derivative) and from dA^n (may be null)
template <int D>
__device__ __forceinline__ void dual_point_A(const PGeom &pg, const int cell[3], const Dual off[3],
                                             const double *__restrict__ A_n,
                                             const double *__restrict__ dA_n, Dual Ax[3]) {
  point_interp<D, Dual>(pg, cell, off, A_n, Ax);
  if (dA_n) {
    const double ov[3] = {off[0].v, off[1].v, off[2].v};
    double dAx[3];
    point_interp<D, double>(pg, cell, ov, dA_n, dAx);
#pragma unroll
    for (int c = 0; c < 3; c++) Ax[c].d += dAx[c];
  }
}

// Dual step start (the first line of Algorithm 1 on dual numbers):
// A^- = A^n_h(x^n), p^n = P^n - q A^-, v^0 = v(p^n)
template <int D>
__global__ void k_dual_step_start(PView<Dual> pv, Dual *Am, Dual *v0,
                                  const double *__restrict__ A_n, const double *__restrict__ dA_n,
                                  PGeom pg, KConst<Dual> kc) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np) return;
  int cell[3] = {0, 0, 0};
  Dual off[3] = {Dual(0.0), Dual(0.0), Dual(0.0)};
  for (int l = 0; l < D; l++) {
    cell[l] = pv.cell[l * pv.cap + i];
    off[l] = pv.off[l * pv.cap + i];
  }
  Dual Ax[3];
  dual_point_A<D>(pg, cell, off, A_n, dA_n, Ax);
  const int s = pv.sp[i];
  const Dual q(pv.w[i] * kc.qs[s]), m(pv.w[i] * kc.ms[s]);
  Dual p[3], p2(0.0);
  for (int c = 0; c < 3; c++) {
    Am[c * pv.cap + i] = Ax[c];
    p[c] = pv.P[c * pv.cap + i] - q * Ax[c];
    p2 += p[c] * p[c];
  }
  const Dual ig = rsqrt(Dual(1.0) + p2 / (m * m * kc.kappa * kc.kappa));
  for (int c = 0; c < 3; c++) v0[c * pv.cap + i] = p[c] / m * ig;
}

// Seed of the particle tangents at the started state: zero offset tangent,
// dP = m du + q (P dA)_h(x); du in load order (3 x n, may be null)
template <int D>
__global__ void k_tangent_seed(int64_t np, int64_t cap, const int32_t *__restrict__ cell_a,
                               const double *__restrict__ off_a, const double *__restrict__ w,
                               const int32_t *__restrict__ sp, const int64_t *__restrict__ id,
                               const double *__restrict__ du, const double *__restrict__ dA,
                               PGeom pg, KConst<double> kc, double *t_off, double *t_P) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  int cell[3] = {0, 0, 0};
  double off[3] = {0.0, 0.0, 0.0};
  for (int l = 0; l < D; l++) {
    cell[l] = cell_a[l * cap + i];
    off[l] = off_a[l * cap + i];
    t_off[l * cap + i] = 0.0;
  }
  double dAx[3] = {0.0, 0.0, 0.0};
  if (dA) point_interp<D, double>(pg, cell, off, dA, dAx);
  const int s = sp[i];
  const double q = w[i] * kc.qs[s], m = w[i] * kc.ms[s];
  const int64_t j = id[i];
  for (int c = 0; c < 3; c++) t_P[c * cap + i] = m * (du ? du[c * np + j] : 0.0) + q * dAx[c];
}

// the particle part of the tangent's commit: x^{n+1} = x^n + dt vbar and
// P <- P^{n+1} differentiate to doff += dt dvbar / dx, dP <- dP^{n+1}
__global__ void k_tangent_commit(int64_t np, int64_t cap, int d, const Dual *__restrict__ vb,
                                 const Dual *__restrict__ Pn, PGeom pg, double dt, double *t_off,
                                 double *t_P) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  for (int l = 0; l < d; l++) t_off[l * cap + i] += dt * vb[l * cap + i].d * pg.inv_dx[l];
  for (int c = 0; c < 3; c++) t_P[c * cap + i] = Pn[c * cap + i].d;
}

// dx (physical units) and dP in load order
__global__ void k_tangent_export(int64_t np, int64_t cap, int d, const int64_t *__restrict__ id,
                                 const double *__restrict__ t_off, const double *__restrict__ t_P,
                                 PGeom pg, double *dx, double *dP) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int64_t j = id[i];
  if (dx)
    for (int l = 0; l < d; l++) dx[l * np + j] = t_off[l * cap + i] * pg.dx[l];
  if (dP)
    for (int c = 0; c < 3; c++) dP[c * np + j] = t_P[c * cap + i];
}

// tangent of the kinetic energy |p|^2 / (m (gamma + 1)), p = P - q A_h(x)
// (Eq. Kkin-nondim), per CTA partial sums in psum
template <int D>
__global__ void __launch_bounds__(kPT)
k_kinetic_tangent(int64_t np, int64_t cap, const int32_t *__restrict__ cell_a,
                  const double *__restrict__ off_a, const double *__restrict__ P_a,
                  const double *__restrict__ w, const int32_t *__restrict__ sp,
                  const double *__restrict__ t_off, const double *__restrict__ t_P,
                  const double *__restrict__ A_n, const double *__restrict__ dA_n, PGeom pg,
                  KConst<double> kc, double *psum) {
  const int64_t i = blockIdx.x * (int64_t)kPT + threadIdx.x;
  double dk = 0.0;
  if (i < np) {
    int cell[3] = {0, 0, 0};
    Dual off[3] = {Dual(0.0), Dual(0.0), Dual(0.0)};
    for (int l = 0; l < D; l++) {
      cell[l] = cell_a[l * cap + i];
      off[l] = Dual(off_a[l * cap + i], t_off[l * cap + i]);
    }
    Dual Ax[3];
    dual_point_A<D>(pg, cell, off, A_n, dA_n, Ax);
    const int s = sp[i];
    const double q = w[i] * kc.qs[s], m = w[i] * kc.ms[s];
    Dual p2(0.0);
    for (int c = 0; c < 3; c++) {
      const Dual p = Dual(P_a[c * cap + i], t_P[c * cap + i]) - Dual(q) * Ax[c];
      p2 += p * p;
    }
    const Dual gam = sqrt(Dual(1.0) + p2 / Dual(m * m * kc.kappa * kc.kappa));
    dk = (p2 / (Dual(m) * (gam + Dual(1.0)))).d;
  }
  for (int o = 16; o > 0; o >>= 1) dk += __shfl_down_sync(0xffffffffu, dk, o);
  __shared__ double sh[kPT / 32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dk;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kPT / 32; k++) t += sh[k];
    psum[blockIdx.x] = t;
  }
}

inline int grid1(int64_t n) { return (int)((n + 255) / 256); }

// dual views of the particle arrays: off, P, Am, v0, vbar, Pnew (dual
// storage pd of (dim + 15) * cap entries), the rest shared with the context
PView<Dual> dual_view(pic_ctx *ctx, Dual *pd) {
  const int d = ctx->g.dim;
  const int64_t cap = ctx->cap;
  PView<Dual> pv;
  pv.np = ctx->np;
  pv.cap = cap;
  pv.cell = ctx->cell;
  pv.off = pd;
  pv.P = pd + (size_t)d * cap;
  pv.Am = pv.P + 3 * cap;
  pv.v0 = pv.Am + 3 * cap;
  pv.vbar = pd + (size_t)(d + 9) * cap;
  pv.Pnew = pv.vbar + 3 * cap;
  pv.w = ctx->w;
  pv.sp = ctx->sp;
  pv.iters = ctx->tmp_i;  // the primal's inner counts stay untouched
  return pv;
}

// the particle map on dual numbers (plain pass: deposit only)
int launch_dual_map(pic_ctx *ctx, const PView<Dual> &pv, const Dual *rec, double *Jd,
                    const KConst<Dual> &kc) {
  if (pv.np == 0) return PIC_OK;
  const PGeom pg = pgeom(ctx);
  const int nb = nblk(pv.np);
  if (ctx->g.dim == 1)
    k_map<1, Dual, false, false><<<nb, kPT, 0, ctx->st>>>(pv, rec, rec, Jd, pg, kc, ctx->cnt_dev,
                                                          ctx->psum, nullptr);
  else if (ctx->g.dim == 2)
    k_map<2, Dual, false, false><<<nb, kPT, 0, ctx->st>>>(pv, rec, rec, Jd, pg, kc, ctx->cnt_dev,
                                                          ctx->psum, nullptr);
  else
    k_map<3, Dual, false, false><<<nb, kPT, 0, ctx->st>>>(pv, rec, rec, Jd, pg, kc, ctx->cnt_dev,
                                                          ctx->psum, nullptr);
  KCHECK();
  return PIC_OK;
}

int launch_dual_step_start(pic_ctx *ctx, const PView<Dual> &pv, const double *dA_n,
                           const KConst<Dual> &kc) {
  if (pv.np == 0) return PIC_OK;
  const PGeom pg = pgeom(ctx);
  Dual *Am = const_cast<Dual *>(pv.Am), *v0 = const_cast<Dual *>(pv.v0);
  const int nb = nblk(pv.np);
  if (ctx->g.dim == 1)
    k_dual_step_start<1><<<nb, kPT, 0, ctx->st>>>(pv, Am, v0, ctx->A_real, dA_n, pg, kc);
  else if (ctx->g.dim == 2)
    k_dual_step_start<2><<<nb, kPT, 0, ctx->st>>>(pv, Am, v0, ctx->A_real, dA_n, pg, kc);
  else
    k_dual_step_start<3><<<nb, kPT, 0, ctx->st>>>(pv, Am, v0, ctx->A_real, dA_n, pg, kc);
  KCHECK();
  return PIC_OK;
}

// read the map's counters; PIC_EINNER if an inner solve failed
int dual_map_status(pic_ctx *ctx, const char *what) {
  EvalCounters cnt;
  CK(cudaMemcpyAsync(&cnt, ctx->cnt_dev, sizeof cnt, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (cnt.status) {
    ctx->err = std::string(what) + ": inner particle solve failed (status bits " +
               std::to_string(cnt.status) + ")";
    return PIC_EINNER;
  }
  return PIC_OK;
}

bool tangent_supported(pic_ctx *ctx, const char *what) {
  if (ctx->rsize != 8 || ctx->opt.order != 2 || ctx->opt.refine_max != 0 ||
      ctx->opt.inner_warm_start) {
    ctx->err = std::string(what) +
               ": FP64, quadratic shapes, no refinement, cold inner start only";
    return false;
  }
  return true;
}

}  // namespace

extern "C" int pic_eval_map_jvp(pic_ctx *ctx, const double *j, const double *dj, double tol,
                                double *H, double *dH, int on_device) {
  if (!ctx || !j || !dj) return PIC_EARG;
  TraceRange trace("pic_eval_map_jvp");
  if (!ctx->started) {
    ctx->err = "pic_eval_map_jvp before pic_start";
    return PIC_ESTATE;
  }
  if (!tangent_supported(ctx, "pic_eval_map_jvp")) return PIC_EARG;
  const int d = ctx->g.dim, Ng = ctx->g.Ng, nvp = node_record_len(d);
  const int64_t cap = ctx->cap;
  const size_t N3 = (size_t)3 * Ng;
  double tr, ta, itr, ita;
  tolerances(ctx, tol, &tr, &ta, &itr, &ita);
  const StepConst sc = make_sc(ctx, itr, ita);
  // scratch: zero modes (also a zero real array), tangent records, dual
  // records, [J_orb | dJ_orb], j and dj, A^{n+1} tangent, dual particles
  const size_t b_zero = sizeof(double2) * N3, b_tan = sizeof(double) * (size_t)Ng * nvp,
               b_rec = sizeof(Dual) * (size_t)Ng * nvp, b_cur = sizeof(double) * 2 * N3,
               b_in = sizeof(double) * 3 * N3, b_par = sizeof(Dual) * (size_t)cap * (d + 15);
  struct Scratch {
    void *p = nullptr;
    ~Scratch() {
      if (p) cudaFree(p);
    }
  } scr;
  CK(cudaMalloc(&scr.p, b_zero + b_tan + b_rec + b_cur + b_in + b_par));
  char *base = (char *)scr.p;
  double2 *zero = (double2 *)base;
  double *tan_rec = (double *)(base + b_zero);
  Dual *rec = (Dual *)(base + b_zero + b_tan);
  double *Jd = (double *)(base + b_zero + b_tan + b_rec);
  double *jin = Jd + 2 * N3, *djin = jin + N3, *dA1 = djin + N3;
  Dual *pd = (Dual *)(base + b_zero + b_tan + b_rec + b_cur + b_in);
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(jin, j, sizeof(double) * N3, kin, ctx->st));
  CK(cudaMemcpyAsync(djin, dj, sizeof(double) * N3, kin, ctx->st));
  CK(cudaMemsetAsync(zero, 0, b_zero, ctx->st));
  CK(cudaMemsetAsync(Jd, 0, b_cur, ctx->st));
  CK(cudaMemsetAsync(ctx->cnt_dev, 0, sizeof(EvalCounters), ctx->st));
  int e;
  if ((e = particles_step_start(ctx))) return e;
  // tangent field step (zero accepted state: A^n does not depend on j), its
  // records kept apart; then the primal field step and records
  const SpecState zs = {zero, zero, zero, zero, zero};
  const SpecState cand = {ctx->rho1_h, ctx->phi1_h, ctx->psi1_h, ctx->A1_h, ctx->U1_h};
  if ((e = field_real_to_complex(ctx, djin, ctx->jh, 3))) return e;
  if ((e = fft_nd(ctx, ctx->jh, 3, -1))) return e;
  if ((e = field_cn_update_into(ctx, ctx->jh, zs, cand, ctx->work_h, 0))) return e;
  if ((e = field_pack_nodes_into(ctx, ctx->work_h, (const double *)zero, dA1, tan_rec))) return e;
  if ((e = field_real_to_complex(ctx, jin, ctx->jh, 3))) return e;
  if ((e = fft_nd(ctx, ctx->jh, 3, -1))) return e;
  if ((e = field_cn_update(ctx, ctx->jh, 0))) return e;
  if ((e = field_pack_nodes(ctx, 0))) return e;
  const int64_t nrec = (int64_t)Ng * nvp;
  k_zip<<<grid1(nrec), 256, 0, ctx->st>>>((const double *)ctx->nodes, tan_rec, rec, nrec, 1, 0,
                                          0);
  KCHECK();
  if (ctx->np > 0) {
    const PView<Dual> pv = dual_view(ctx, pd);
    Dual *off_d = const_cast<Dual *>(pv.off), *P_d = const_cast<Dual *>(pv.P),
         *Am_d = const_cast<Dual *>(pv.Am), *v0_d = const_cast<Dual *>(pv.v0);
    // particle inputs with zero tangent (the state does not depend on j)
    k_zip<<<grid1(ctx->np), 256, 0, ctx->st>>>((const double *)ctx->off, nullptr, off_d, ctx->np,
                                               d, cap, cap);
    KCHECK();
    k_zip<<<grid1(ctx->np), 256, 0, ctx->st>>>((const double *)ctx->P, nullptr, P_d, ctx->np, 3,
                                               cap, cap);
    KCHECK();
    k_zip<<<grid1(ctx->np), 256, 0, ctx->st>>>((const double *)ctx->Am, nullptr, Am_d, ctx->np,
                                               3, cap, cap);
    KCHECK();
    k_zip<<<grid1(ctx->np), 256, 0, ctx->st>>>((const double *)ctx->v0, nullptr, v0_d, ctx->np,
                                               3, cap, cap);
    KCHECK();
    if ((e = launch_dual_map(ctx, pv, rec, Jd, kconst<Dual>(sc, pgeom(ctx))))) return e;
  }
  // H = P J_orb and dH = P dJ_orb
  if ((e = field_project_real(ctx, Jd, Jd, 3))) return e;
  if ((e = field_project_real(ctx, Jd + N3, Jd + N3, 3))) return e;
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (H) CK(cudaMemcpyAsync(H, Jd, sizeof(double) * N3, kout, ctx->st));
  if (dH) CK(cudaMemcpyAsync(dH, Jd + N3, sizeof(double) * N3, kout, ctx->st));
  return dual_map_status(ctx, "pic_eval_map_jvp");
}

// ------------------------------------------------------------ step tangent
void tangent_free(pic_ctx *ctx) {
  if (!ctx || !ctx->tan) return;
  if (ctx->tan->block) cudaFree(ctx->tan->block);
  delete ctx->tan;
  ctx->tan = nullptr;
}

namespace {

// A tangent state with its scratch, all zero (a zero state tangent), not
// attached to the context; null (ctx->err set) if the allocation fails.
TangentState *tangent_state_new(pic_ctx *ctx) {
  const size_t d = ctx->g.dim, Ng = ctx->g.Ng, nvp = node_record_len((int)d);
  const size_t cap = ctx->cap, N3 = 3 * Ng;
  const size_t C = sizeof(double2), R = sizeof(double), Q = sizeof(Dual);
  // sizes of the parts, each rounded up to 256 bytes
  const size_t parts[] = {R * d * cap, R * 3 * cap,           // off, P
                          C * 9 * Ng,  C * 9 * Ng,            // f, f1
                          R * N3,      R * N3,                // A_real, A1_real
                          C * N3,      C * (d + 3) * Ng,      // jh, work
                          R * Ng * nvp, Q * Ng * nvp,         // rec, drec
                          Q * (d + 15) * cap, R * 2 * N3,     // dpart, Jd
                          R * (kKrylov + 1) * N3,             // V
                          R * N3, R * N3, R * N3, R * N3};    // x, b, w, Tx
  size_t off[sizeof parts / sizeof parts[0] + 1] = {0};
  const int np_ = (int)(sizeof parts / sizeof parts[0]);
  for (int k = 0; k < np_; k++) off[k + 1] = off[k] + (parts[k] + 255) / 256 * 256;
  TangentState *t = new TangentState();
  if (cudaMalloc(&t->block, off[np_]) != cudaSuccess) {
    cudaGetLastError();
    delete t;
    ctx->err = "tangent state: device allocation failed";
    return nullptr;
  }
  char *b = (char *)t->block;
  t->off = (double *)(b + off[0]);
  t->P = (double *)(b + off[1]);
  double2 *f = (double2 *)(b + off[2]), *f1 = (double2 *)(b + off[3]);
  t->f = {f, f + Ng, f + 2 * Ng, f + 3 * Ng, f + 6 * Ng};
  t->f1 = {f1, f1 + Ng, f1 + 2 * Ng, f1 + 3 * Ng, f1 + 6 * Ng};
  t->A_real = (double *)(b + off[4]);
  t->A1_real = (double *)(b + off[5]);
  t->jh = (double2 *)(b + off[6]);
  t->work = (double2 *)(b + off[7]);
  t->rec = (double *)(b + off[8]);
  t->drec = b + off[9];
  t->dpart = b + off[10];
  t->Jd = (double *)(b + off[11]);
  t->V = (double *)(b + off[12]);
  t->x = (double *)(b + off[13]);
  t->b = (double *)(b + off[14]);
  t->w = (double *)(b + off[15]);
  t->Tx = (double *)(b + off[16]);
  t->gmres_iters = 0;
  if (cudaMemsetAsync(t->block, 0, off[np_], ctx->st) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(t->block);
    delete t;
    ctx->err = "tangent state: clearing failed";
    return nullptr;
  }
  return t;
}

void tangent_state_delete(TangentState *t) {
  if (!t) return;
  if (t->block) cudaFree(t->block);
  delete t;
}

int tangent_alloc(pic_ctx *ctx) {
  TangentState *t = tangent_state_new(ctx);
  if (!t) return PIC_ENOMEM;
  ctx->tan = t;
  return PIC_OK;
}

// The tangent map of one step at its converged current (records of the
// primal in ctx->nodes): out = P dJ_orb for the tangent trial current v and
// the state tangent; the tangent candidates f1, A1_real and the dual vbar,
// Pnew of the particles are those of v afterwards.
int tangent_eval(pic_ctx *ctx, TangentState &t, const PView<Dual> &pv, const KConst<Dual> &kc,
                 const double *v, double *out) {
  const int Ng = ctx->g.Ng, nvp = node_record_len(ctx->g.dim);
  const size_t N3 = (size_t)3 * Ng;
  int e;
  if ((e = field_real_to_complex(ctx, v, t.jh, 3))) return e;
  if ((e = fft_nd(ctx, t.jh, 3, -1))) return e;
  if ((e = field_cn_update_into(ctx, t.jh, t.f, t.f1, t.work, 0))) return e;
  if ((e = field_pack_nodes_into(ctx, t.work, t.A_real, t.A1_real, t.rec))) return e;
  const int64_t nrec = (int64_t)Ng * nvp;
  k_zip<<<grid1(nrec), 256, 0, ctx->st>>>((const double *)ctx->nodes, t.rec, (Dual *)t.drec,
                                          nrec, 1, 0, 0);
  KCHECK();
  CK(cudaMemsetAsync(t.Jd, 0, sizeof(double) * 2 * N3, ctx->st));
  CK(cudaMemsetAsync(ctx->cnt_dev, 0, sizeof(EvalCounters), ctx->st));
  if ((e = launch_dual_map(ctx, pv, (const Dual *)t.drec, t.Jd, kc))) return e;
  if ((e = field_project_real(ctx, t.Jd + N3, out, 3))) return e;
  return dual_map_status(ctx, "tangent step");
}

double norm2(pic_ctx *ctx, const double *a, int *err) {
  double v = 0.0;
  const double *pa[1] = {a};
  *err = dots(ctx, pa, pa, 1, &v);
  return std::sqrt(v);
}

}  // namespace

// Restarted GMRES(kKrylov) for (I - A) x = b, where T(v) = A v + b is the
// tangent map (affine in v): b = T(0) and (I - A) v = v - T(v) + b.  The
// basis is orthogonalised by classical Gram-Schmidt with one
// re-orthogonalisation; the small least-squares problem is solved on the
// host by Givens rotations.  Every restart ends with the true residual
// T(x) - x, so that the last tangent evaluation is the one at x.
int tangent_solve(pic_ctx *ctx, const StepConst &sc, double tol) {
  TraceRange trace("tangent_solve");
  TangentState &t = *ctx->tan;
  const size_t N3 = (size_t)3 * ctx->g.Ng;
  const KConst<Dual> kc = kconst<Dual>(sc, pgeom(ctx));
  const PView<Dual> pv = dual_view(ctx, (Dual *)t.dpart);
  int e;
  // dual particle inputs at x^n and the dual step start
  if (ctx->np > 0) {
    Dual *off_d = const_cast<Dual *>(pv.off), *P_d = const_cast<Dual *>(pv.P);
    k_zip<<<grid1(ctx->np), 256, 0, ctx->st>>>((const double *)ctx->off, t.off, off_d, ctx->np,
                                               ctx->g.dim, ctx->cap, ctx->cap);
    KCHECK();
    k_zip<<<grid1(ctx->np), 256, 0, ctx->st>>>((const double *)ctx->P, t.P, P_d, ctx->np, 3,
                                               ctx->cap, ctx->cap);
    KCHECK();
    if ((e = launch_dual_step_start(ctx, pv, t.A_real, kc))) return e;
  }
  const double rtol = std::fmax(tol, 1e-12);
  t.gmres_iters = 0;
  CK(cudaMemsetAsync(t.x, 0, sizeof(double) * N3, ctx->st));
  if ((e = tangent_eval(ctx, t, pv, kc, t.x, t.b))) return e;  // b = T(0)
  const double bn = norm2(ctx, t.b, &e);
  if (e) return e;
  if (!std::isfinite(bn)) {
    ctx->err = "tangent step: the tangent map is not finite";
    return PIC_EOUTER;
  }
  if (bn == 0.0) return PIC_OK;  // x = 0, and the last evaluation was T(0)
  // r = T(x) - x = b for x = 0, kept in V_0
  double *V0 = t.V;
  CK(cudaMemcpyAsync(V0, t.b, sizeof(double) * N3, cudaMemcpyDeviceToDevice, ctx->st));
  double beta = bn, ref = bn, beta_prev = bn;
  std::string hist;  // relative residual after each restart
  const int m = kKrylov;
  for (int restart = 0; restart < kRestarts; restart++) {
    if (restart > 0 && beta <= rtol * ref) return PIC_OK;
    if ((e = lincomb(ctx, V0, V0, 1.0 / beta, V0, 0.0, N3))) return e;
    std::vector<double> H((m + 1) * m, 0.0), g(m + 1, 0.0), cs(m, 0.0), sn(m, 0.0);
    g[0] = beta;
    int kk = 0;
    for (int k = 0; k < m; k++) {
      double *Vk = t.V + (size_t)k * N3, *Vn = t.V + (size_t)(k + 1) * N3;
      // w = V_k - T(V_k) + b
      if ((e = tangent_eval(ctx, t, pv, kc, Vk, t.w))) return e;
      if ((e = lincomb(ctx, t.w, Vk, 1.0, t.w, -1.0, N3))) return e;
      if ((e = lincomb(ctx, t.w, t.w, 1.0, t.b, 1.0, N3))) return e;
      t.gmres_iters++;
      for (int pass = 0; pass < 2; pass++) {
        const double *pa[kKrylov + 1], *pb[kKrylov + 1];
        double h[kKrylov + 1];
        for (int i = 0; i <= k; i++) {
          pa[i] = t.V + (size_t)i * N3;
          pb[i] = t.w;
        }
        if ((e = dots(ctx, pa, pb, k + 1, h))) return e;
        for (int i = 0; i <= k; i++) {
          H[i * m + k] += h[i];
          if ((e = lincomb(ctx, t.w, t.w, 1.0, pa[i], -h[i], N3))) return e;
        }
      }
      const double hn = norm2(ctx, t.w, &e);
      if (e) return e;
      if (!std::isfinite(hn)) {
        ctx->err = "tangent step: non-finite Krylov vector";
        return PIC_EOUTER;
      }
      H[(k + 1) * m + k] = hn;
      // previous rotations, then the one that zeroes H[k+1][k]
      for (int i = 0; i < k; i++) {
        const double a = H[i * m + k], c = H[(i + 1) * m + k];
        H[i * m + k] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + k] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[k * m + k], c = H[(k + 1) * m + k];
      const double rr = std::hypot(a, c);
      cs[k] = rr > 0.0 ? a / rr : 1.0;
      sn[k] = rr > 0.0 ? c / rr : 0.0;
      H[k * m + k] = rr;
      H[(k + 1) * m + k] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      kk = k + 1;
      if (hn > 0.0 && (e = lincomb(ctx, Vn, t.w, 1.0 / hn, t.w, 0.0, N3))) return e;
      if (std::fabs(g[k + 1]) <= 0.5 * rtol * ref || hn == 0.0) break;
    }
    // y from the triangular system, x += V y
    std::vector<double> y(kk, 0.0);
    for (int i = kk - 1; i >= 0; i--) {
      double s = g[i];
      for (int q = i + 1; q < kk; q++) s -= H[i * m + q] * y[q];
      y[i] = H[i * m + i] != 0.0 ? s / H[i * m + i] : 0.0;
    }
    for (int i = 0; i < kk; i++)
      if ((e = lincomb(ctx, t.x, t.x, 1.0, t.V + (size_t)i * N3, y[i], N3))) return e;
    // true residual r = T(x) - x into V_0, measured against the larger of
    // |b| and |x| (the solution may be larger than the right-hand side)
    if ((e = tangent_eval(ctx, t, pv, kc, t.x, t.Tx))) return e;
    if ((e = lincomb(ctx, V0, t.Tx, 1.0, t.x, -1.0, N3))) return e;
    beta = norm2(ctx, V0, &e);
    if (e) return e;
    ref = std::fmax(bn, norm2(ctx, t.x, &e));
    if (e) return e;
    char buf[32];
    std::snprintf(buf, sizeof buf, "%s%.3e", hist.empty() ? "" : ", ", beta / ref);
    hist += buf;
    if (!std::isfinite(beta)) break;
    if (beta > rtol * ref && beta > 0.5 * beta_prev && beta <= kNoiseFloor * ref) return PIC_OK;
    beta_prev = beta;
  }
  if (beta <= rtol * ref) return PIC_OK;
  ctx->err = "tangent step: GMRES did not reach the tolerance (relative residuals " + hist +
             ")";
  return PIC_EOUTER;
}

// ---------------------------------------------------------- Newton-Krylov
// The Newton direction of the outer equation H(j) - j = 0 at the current
// iterate, for the Newton-Krylov alternative to Algorithm 1's Anderson
// iteration: (I - H'(j)) delta = r by GMRES(kKrylov) with up to two
// restarts, to the relative residual eta (an inexact Newton step).  H'(j) v
// is the tangent map with a zero state tangent: one dual map evaluation at
// the gather records of the last plain evaluation (those of j).
struct NkState {
  TangentState *t;
  PView<Dual> pv;
  KConst<Dual> kc;
};

int nk_begin(pic_ctx *ctx, const StepConst &sc, NkState **out) {
  *out = nullptr;
  TangentState *t = tangent_state_new(ctx);
  if (!t) return PIC_ENOMEM;
  NkState *nk = new NkState();
  nk->t = t;
  nk->kc = kconst<Dual>(sc, pgeom(ctx));
  nk->pv = dual_view(ctx, (Dual *)t->dpart);
  *out = nk;
  int e;
  if (ctx->np > 0) {  // the particle inputs with zero tangents, and the dual step start
    Dual *off_d = const_cast<Dual *>(nk->pv.off), *P_d = const_cast<Dual *>(nk->pv.P);
    k_zip<<<grid1(ctx->np), 256, 0, ctx->st>>>((const double *)ctx->off, nullptr, off_d, ctx->np,
                                               ctx->g.dim, ctx->cap, ctx->cap);
    KCHECK();
    k_zip<<<grid1(ctx->np), 256, 0, ctx->st>>>((const double *)ctx->P, nullptr, P_d, ctx->np, 3,
                                               ctx->cap, ctx->cap);
    KCHECK();
    if ((e = launch_dual_step_start(ctx, nk->pv, nullptr, nk->kc))) return e;
  }
  return PIC_OK;
}

void nk_end(NkState *nk) {
  if (!nk) return;
  tangent_state_delete(nk->t);
  delete nk;
}

int nk_direction(pic_ctx *ctx, NkState *nk, const double *r, double eta, double *x, int *iters) {
  TraceRange trace("newton_direction");
  TangentState &t = *nk->t;
  const size_t N3 = (size_t)3 * ctx->g.Ng;
  const int m = kKrylov;
  int e;
  *iters = 0;
  CK(cudaMemsetAsync(x, 0, sizeof(double) * N3, ctx->st));
  double *V0 = t.V;
  CK(cudaMemcpyAsync(V0, r, sizeof(double) * N3, cudaMemcpyDeviceToDevice, ctx->st));
  double beta = norm2(ctx, V0, &e);
  if (e) return e;
  const double ref = beta;
  if (!(beta > 0.0)) return PIC_OK;
  for (int restart = 0; restart < 3; restart++) {
    if ((e = lincomb(ctx, V0, V0, 1.0 / beta, V0, 0.0, N3))) return e;
    std::vector<double> H((m + 1) * m, 0.0), g(m + 1, 0.0), cs(m, 0.0), sn(m, 0.0);
    g[0] = beta;
    int kk = 0;
    for (int k = 0; k < m; k++) {
      double *Vk = t.V + (size_t)k * N3, *Vn = t.V + (size_t)(k + 1) * N3;
      // w = V_k - H'(j) V_k
      if ((e = tangent_eval(ctx, t, nk->pv, nk->kc, Vk, t.w))) return e;
      if ((e = lincomb(ctx, t.w, Vk, 1.0, t.w, -1.0, N3))) return e;
      (*iters)++;
      for (int pass = 0; pass < 2; pass++) {
        const double *pa[kKrylov + 1], *pb[kKrylov + 1];
        double h[kKrylov + 1];
        for (int i = 0; i <= k; i++) {
          pa[i] = t.V + (size_t)i * N3;
          pb[i] = t.w;
        }
        if ((e = dots(ctx, pa, pb, k + 1, h))) return e;
        for (int i = 0; i <= k; i++) {
          H[i * m + k] += h[i];
          if ((e = lincomb(ctx, t.w, t.w, 1.0, pa[i], -h[i], N3))) return e;
        }
      }
      const double hn = norm2(ctx, t.w, &e);
      if (e) return e;
      if (!std::isfinite(hn)) {
        ctx->err = "Newton direction: non-finite Krylov vector";
        return PIC_EOUTER;
      }
      H[(k + 1) * m + k] = hn;
      for (int i = 0; i < k; i++) {
        const double a = H[i * m + k], c = H[(i + 1) * m + k];
        H[i * m + k] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + k] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[k * m + k], c = H[(k + 1) * m + k];
      const double rr = std::hypot(a, c);
      cs[k] = rr > 0.0 ? a / rr : 1.0;
      sn[k] = rr > 0.0 ? c / rr : 0.0;
      H[k * m + k] = rr;
      H[(k + 1) * m + k] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      kk = k + 1;
      if (hn > 0.0 && (e = lincomb(ctx, Vn, t.w, 1.0 / hn, t.w, 0.0, N3))) return e;
      if (std::fabs(g[k + 1]) <= eta * ref || hn == 0.0) break;
    }
    std::vector<double> y(kk, 0.0);
    for (int i = kk - 1; i >= 0; i--) {
      double s = g[i];
      for (int q = i + 1; q < kk; q++) s -= H[i * m + q] * y[q];
      y[i] = H[i * m + i] != 0.0 ? s / H[i * m + i] : 0.0;
    }
    for (int i = 0; i < kk; i++)
      if ((e = lincomb(ctx, x, x, 1.0, t.V + (size_t)i * N3, y[i], N3))) return e;
    if (std::fabs(g[kk]) <= eta * ref) return PIC_OK;
    // restart from the true residual r - (x - H'(j) x)
    if ((e = tangent_eval(ctx, t, nk->pv, nk->kc, x, t.Tx))) return e;
    (*iters)++;
    if ((e = lincomb(ctx, V0, r, 1.0, x, -1.0, N3))) return e;
    if ((e = lincomb(ctx, V0, V0, 1.0, t.Tx, 1.0, N3))) return e;
    beta = norm2(ctx, V0, &e);
    if (e) return e;
    if (!std::isfinite(beta)) {
      ctx->err = "Newton direction: non-finite residual";
      return PIC_EOUTER;
    }
    if (beta <= eta * ref) return PIC_OK;
  }
  return PIC_OK;  // an inexact direction; the backtracking decides
}

int tangent_commit(pic_ctx *ctx) {
  TangentState &t = *ctx->tan;
  if (ctx->np > 0) {
    const PView<Dual> pv = dual_view(ctx, (Dual *)t.dpart);
    k_tangent_commit<<<grid1(ctx->np), 256, 0, ctx->st>>>(ctx->np, ctx->cap, ctx->g.dim, pv.vbar,
                                                          pv.Pnew, pgeom(ctx), ctx->dt, t.off,
                                                          t.P);
    KCHECK();
  }
  std::swap(t.f, t.f1);
  std::swap(t.A_real, t.A1_real);
  return PIC_OK;
}

extern "C" int pic_tangent_begin(pic_ctx *ctx, const double *du, const double *dA,
                                 const double *dU, int on_device) {
  if (!ctx) return PIC_EARG;
  if (!ctx->started) {
    ctx->err = "pic_tangent_begin before pic_start";
    return PIC_ESTATE;
  }
  if (!tangent_supported(ctx, "pic_tangent_begin")) return PIC_EARG;
  tangent_free(ctx);
  int e;
  if ((e = tangent_alloc(ctx))) return e;
  TangentState &t = *ctx->tan;
  const int Ng = ctx->g.Ng;
  const size_t N3 = (size_t)3 * Ng;
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // the potentials' seed, projected as pic_start projects A^0 and U^0; dA back
  // to real space for the gathers
  if (dA) CK(cudaMemcpyAsync(t.A_real, dA, sizeof(double) * N3, kin, ctx->st));
  if (dU) CK(cudaMemcpyAsync(t.A1_real, dU, sizeof(double) * N3, kin, ctx->st));
  if ((e = field_real_to_complex(ctx, t.A_real, t.f.A, 3))) return e;
  if ((e = fft_nd(ctx, t.f.A, 3, -1))) return e;
  if ((e = field_project_h(ctx, t.f.A, 3))) return e;
  if ((e = field_real_to_complex(ctx, t.A1_real, t.f.U, 3))) return e;
  if ((e = fft_nd(ctx, t.f.U, 3, -1))) return e;
  if ((e = field_project_h(ctx, t.f.U, 3))) return e;
  CK(cudaMemcpyAsync(t.work, t.f.A, sizeof(double2) * N3, cudaMemcpyDeviceToDevice, ctx->st));
  if ((e = fft_nd(ctx, t.work, 3, +1))) return e;
  if ((e = field_complex_to_real(ctx, t.work, t.A_real, 3, 1.0 / Ng))) return e;
  // drho = 0 (the positions carry no seed); dphi from Gauss, dpsi from Lorenz
  CK(cudaMemsetAsync(t.f.rho, 0, sizeof(double2) * Ng, ctx->st));
  if ((e = field_initial_constraints_into(ctx, t.f))) return e;
  // particles: zero offset tangent, dP = m du + q (P dA)_h(x)
  if (ctx->np > 0) {
    const double *du_dev = nullptr;
    if (du) {
      if (on_device) {
        du_dev = du;
      } else {
        CK(cudaMemcpyAsync(ctx->tmp_d, du, sizeof(double) * 3 * ctx->np, cudaMemcpyHostToDevice,
                           ctx->st));
        du_dev = ctx->tmp_d;
      }
    }
    const PGeom pg = pgeom(ctx);
    const KConst<double> kc = kconst<double>(make_sc(ctx, 0.0, 0.0), pg);
    const int nb = grid1(ctx->np);
#define PIC_SEED(DD)                                                                          \
  k_tangent_seed<DD><<<nb, 256, 0, ctx->st>>>(ctx->np, ctx->cap, ctx->cell,                    \
                                              (const double *)ctx->off, ctx->w, ctx->sp, ctx->id, \
                                              du_dev, t.A_real, pg, kc, t.off, t.P)
    if (ctx->g.dim == 1) PIC_SEED(1);
    else if (ctx->g.dim == 2) PIC_SEED(2);
    else PIC_SEED(3);
#undef PIC_SEED
    KCHECK();
  }
  CK(cudaStreamSynchronize(ctx->st));
  return PIC_OK;
}

extern "C" int pic_tangent_end(pic_ctx *ctx) {
  if (!ctx) return PIC_EARG;
  tangent_free(ctx);
  return PIC_OK;
}

extern "C" int pic_get_tangent(pic_ctx *ctx, double *dx, double *dP, double *dA, double *dU,
                               double *dK, double *dW, int *gmres_iters, int on_device) {
  if (!ctx) return PIC_EARG;
  if (!ctx->tan) {
    ctx->err = "pic_get_tangent without pic_tangent_begin";
    return PIC_ESTATE;
  }
  TangentState &t = *ctx->tan;
  const int d = ctx->g.dim, Ng = ctx->g.Ng;
  const int64_t n = ctx->np;
  const size_t N3 = (size_t)3 * Ng;
  const PGeom pg = pgeom(ctx);
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  int e;
  if ((dx || dP) && n > 0) {
    double *ox = dx, *oP = dP;
    if (!on_device) {  // staged in the context's export scratch
      ox = dx ? ctx->tmp_d : nullptr;
      oP = dP ? ctx->tmp_d + 3 * ctx->cap : nullptr;
    }
    k_tangent_export<<<grid1(n), 256, 0, ctx->st>>>(n, ctx->cap, d, ctx->id, t.off, t.P, pg, ox,
                                                    oP);
    KCHECK();
    if (!on_device) {
      if (dx) CK(cudaMemcpyAsync(dx, ox, sizeof(double) * d * n, kout, ctx->st));
      if (dP) CK(cudaMemcpyAsync(dP, oP, sizeof(double) * 3 * n, kout, ctx->st));
    }
  }
  if (dA) CK(cudaMemcpyAsync(dA, t.A_real, sizeof(double) * N3, kout, ctx->st));
  if (dU) {
    CK(cudaMemcpyAsync(t.work, t.f.U, sizeof(double2) * N3, cudaMemcpyDeviceToDevice, ctx->st));
    if ((e = fft_nd(ctx, t.work, 3, +1))) return e;
    if ((e = field_complex_to_real(ctx, t.work, t.w, 3, 1.0 / Ng))) return e;
    CK(cudaMemcpyAsync(dU, t.w, sizeof(double) * N3, kout, ctx->st));
  }
  if (dK) {
    double s = 0.0;
    if (n > 0) {
      const KConst<double> kc = kconst<double>(make_sc(ctx, 0.0, 0.0), pg);
      const int nb = nblk(n);
#define PIC_KT(DD)                                                                          \
  k_kinetic_tangent<DD><<<nb, kPT, 0, ctx->st>>>(n, ctx->cap, ctx->cell,                     \
                                                 (const double *)ctx->off,                   \
                                                 (const double *)ctx->P, ctx->w, ctx->sp,    \
                                                 t.off, t.P, ctx->A_real, t.A_real, pg, kc, \
                                                 ctx->psum)
      if (d == 1) PIC_KT(1);
      else if (d == 2) PIC_KT(2);
      else PIC_KT(3);
#undef PIC_KT
      KCHECK();
      CK(cudaMemcpyAsync(ctx->psum_host, ctx->psum, sizeof(double) * nb, cudaMemcpyDeviceToHost,
                         ctx->st));
      CK(cudaStreamSynchronize(ctx->st));
      for (int b = 0; b < nb; b++) s += ctx->psum_host[b];  // fixed order
    }
    *dK = s;
  }
  if (dW) {
    const SpecState acc = {ctx->rho_h, ctx->phi_h, ctx->psi_h, ctx->A_h, ctx->U_h};
    if ((e = field_energy_tangent(ctx, acc, t.f, dW))) return e;
  }
  if (gmres_iters) *gmres_iters = t.gmres_iters;
  CK(cudaStreamSynchronize(ctx->st));
  return PIC_OK;
}
