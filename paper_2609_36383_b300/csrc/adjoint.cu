// adjoint.cu -- pic_eval_map_vjp(): the adjoint of one evaluation of the
// outer map H(j) = P J_orb(j) (Sec. 4.5), jbar = H'(j)^T ybar, the
// vector-Jacobian product a gradient with respect to the trial current needs.
// The paper differentiates nothing; this is the transpose of the map that
// pic_eval_map_jvp differentiates forward.
//
// H is a composition, transposed from the output back:
//  * P, the Nyquist projector, is symmetric: Jbar = P ybar;
//  * the orbit deposit J = sum_p q vbar_p Sbar_p(vbar_p) / dV depends on the
//    orbit velocity only, and its transpose is the orbit gather of Jbar with
//    the deposit's weights: the per-particle scalar
//    s_p(vbar) = q vbar . G(Jbar; vbar) / dV has gradient gs_p;
//  * the inner Picard fixed point vbar = Phi(vbar, F) (Sec. 4.5) over the
//    gather records F transposes by implicit differentiation: the particle's
//    cotangent lambda solves (I - Phi_vbar^T) lambda = gs (3 x 3), and
//    Phi_F^T lambda is the push's transpose-vector product on the gathered
//    quantities (grad phi^{1/2}, D_i A, A^{n+1} at the orbit's end), scattered
//    to the records with the gather's own orbit weights (a deposit);
//  * the records depend on j through the CN field step, mode by mode a real
//    symmetric map, transposed in field.cu (k_cn_adjoint) between a forward
//    and an inverse transform.
// The particle part runs as three passes, each a kernel: Phi_vbar (three
// sweeps on dual numbers, dual.cuh, at the converged velocity), then gs and
// lambda, then the push's derivatives (one dual push per gathered quantity)
// and the scatters (FP64 atomics).
#include "adjoint_device.cuh"
#include "trace.cuh"

#include <cmath>
#include <string>

namespace {

// Pass 1, one thread per particle: converge vbar as the map does (cold
// start), then Phi_vbar, column e from one inner sweep on dual numbers with
// the velocity seeded along e.  Stores vbar (3 x cap) and Phi_vbar (9 x cap).
template <int D>
__global__ void k_vjp_phi(PView<double> pv, const double *__restrict__ nodes,
                          const Dual *__restrict__ dnodes, PGeom pg, KConst<double> kc,
                          KConst<Dual> kcd, double *__restrict__ vb_out,
                          double *__restrict__ jv_out, EvalCounters *__restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np) return;
  const MapScale<double> ms = {{kc.inv_dx[0], kc.inv_dx[1], kc.inv_dx[2]}, kc.inv_dV};
  const MapScale<Dual> msd = {{kcd.inv_dx[0], kcd.inv_dx[1], kcd.inv_dx[2]}, kcd.inv_dV};
  PushConst<double> pc;
  int cell[3];
  double off[3], dtdx[3], vb[3], Pn1[3];
  vjp_particle<D>(pv, i, kc, ms, pc, cell, off, dtdx);
  for (int c = 0; c < 3; c++) {
    vb[c] = pv.v0[c * pv.cap + i];
    Pn1[c] = pc.Pn[c];
  }
  int it = 0, npieces = 0;
  unsigned int st = 0;
  if (!picard<D, double, false>(pc, cell, off, dtdx, 0.0, 1.0, nodes, pg, kc, ms, vb, Pn1, it,
                                npieces, st, 2)) {
    atomicOr(&cnt->status, st ? st : PIC_ST_NOCONV);
    return;
  }
  const PushConst<Dual> pd = dual_push_const(pc);
  Dual offd[3], dtdxd[3];
  for (int l = 0; l < 3; l++) {
    offd[l] = Dual(off[l]);
    dtdxd[l] = Dual(dtdx[l]);
  }
  for (int e = 0; e < 3; e++) {
    Dual vbd[3];
    for (int l = 0; l < 3; l++) vbd[l] = Dual(vb[l], l == e ? 1.0 : 0.0);
    Dual gphi[3], Dm[3][3], Ap[3];
    int np_ = 0;
    if (!orbit_gather<D, Dual, false>(cell, offd, dtdxd, Dual(0.0), Dual(1.0), dnodes, pg, kcd,
                                      msd, vbd, gphi, Dm, Ap, np_, 2)) {
      atomicOr(&cnt->status, PIC_ST_PIECES);
      return;
    }
    Dual vn[3], Pc[3];
    gmhc_push<D, Dual>(pd, Ap, gphi, Dm, vbd, vn, Pc);
    for (int c = 0; c < 3; c++) jv_out[(size_t)(c * 3 + e) * pv.cap + i] = vn[c].d;
  }
  for (int c = 0; c < 3; c++) vb_out[(size_t)c * pv.cap + i] = vb[c];
}

// Pass 2: the gradient gs of the deposit's scalar s(vbar) = q vbar . G(Jbar;
// vbar) / dV (three orbit gathers on dual numbers) and lambda from
// (I - Phi_vbar^T) lambda = gs.  Stores lambda (3 x cap).
template <int D>
__global__ void k_vjp_lambda(PView<double> pv, const double *__restrict__ Jbar, PGeom pg,
                             KConst<double> kc, KConst<Dual> kcd,
                             const double *__restrict__ vb_in, const double *__restrict__ jv_in,
                             double *__restrict__ lam_out, EvalCounters *__restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np || cnt->status) return;
  const MapScale<double> ms = {{kc.inv_dx[0], kc.inv_dx[1], kc.inv_dx[2]}, kc.inv_dV};
  PushConst<double> pc;
  int cell[3];
  double off[3], dtdx[3], vb[3], Jv[3][3], gs[3];
  vjp_particle<D>(pv, i, kc, ms, pc, cell, off, dtdx);
  for (int c = 0; c < 3; c++) {
    vb[c] = vb_in[(size_t)c * pv.cap + i];
    for (int e = 0; e < 3; e++) Jv[c][e] = jv_in[(size_t)(c * 3 + e) * pv.cap + i];
  }
  const Dual qdv(pc.q * ms.inv_dV);
  for (int e = 0; e < 3; e++) {
    OrbitDot<D, Dual> od;
    od.F = Jbar;
    od.pg = &pg;
    od.kc = &kcd;
    od.order = 2;
    Dual vbd[3];
    for (int l = 0; l < 3; l++) {
      vbd[l] = Dual(vb[l], l == e ? 1.0 : 0.0);
      od.cell[l] = cell[l];
      od.off[l] = Dual(off[l]);
      od.del[l] = vbd[l] * Dual(dtdx[l]);
      od.G[l] = Dual(0.0);
    }
    if (!walk_orbit<D, Dual>(od.off, od.del, od, 2)) {
      atomicOr(&cnt->status, PIC_ST_PIECES);
      return;
    }
    Dual sv(0.0);
    for (int c = 0; c < 3; c++) sv += qdv * vbd[c] * od.G[c];
    gs[e] = sv.d;
  }
  double lam[3];
  if (!solve_adjoint3(Jv, gs, lam)) {
    atomicOr(&cnt->status, PIC_ST_NONFINITE);
    return;
  }
  for (int c = 0; c < 3; c++) lam_out[(size_t)c * pv.cap + i] = lam[c];
}

// Pass 3: the push's transpose-vector product lambda^T dPhi/dg on the
// gathered quantities g at vbar (one dual push per quantity), scattered to
// Fbar with the gather's orbit weights (D_i A's columns were scaled by 1/dx).
template <int D>
__global__ void k_vjp_scatter(PView<double> pv, const double *__restrict__ nodes,
                              const double *__restrict__ vb_in,
                              const double *__restrict__ lam_in, double *__restrict__ Fbar,
                              PGeom pg, KConst<double> kc, const EvalCounters *__restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np || cnt->status) return;
  const MapScale<double> ms = {{kc.inv_dx[0], kc.inv_dx[1], kc.inv_dx[2]}, kc.inv_dV};
  PushConst<double> pc;
  int cell[3];
  double off[3], dtdx[3], vb[3], lam[3];
  vjp_particle<D>(pv, i, kc, ms, pc, cell, off, dtdx);
  for (int c = 0; c < 3; c++) {
    vb[c] = vb_in[(size_t)c * pv.cap + i];
    lam[c] = lam_in[(size_t)c * pv.cap + i];
  }
  const PushConst<Dual> pd = dual_push_const(pc);
  double gphi0[3], Dm0[3][3], Ap0[3];
  int np2 = 0;
  // an orbit too long for the walk was flagged by the first pass (and no
  // pass after it runs then); never use gathered values it did not write
  if (!orbit_gather<D, double, false>(cell, off, dtdx, 0.0, 1.0, nodes, pg, kc, ms, vb, gphi0,
                                      Dm0, Ap0, np2, 2))
    return;
  Dual vbc[3];
  for (int l = 0; l < 3; l++) vbc[l] = Dual(vb[l]);
  double ggphi[3] = {0.0, 0.0, 0.0}, gDm[3][3] = {{0.0}}, gAp[3] = {0.0, 0.0, 0.0};
  const int nin = D + 3 * D + 3;  // grad phi (D), D_i A (3 x D), A^{n+1} (3)
  for (int q = 0; q < nin; q++) {
    Dual gphi[3], Dm[3][3], Ap[3];
    for (int c = 0; c < 3; c++) {
      gphi[c] = Dual(gphi0[c]);
      Ap[c] = Dual(Ap0[c]);
      for (int j = 0; j < 3; j++) Dm[c][j] = Dual(Dm0[c][j]);
    }
    if (q < D) gphi[q].d = 1.0;
    else if (q < 4 * D) Dm[(q - D) / D][(q - D) % D].d = 1.0;
    else Ap[q - 4 * D].d = 1.0;
    Dual vn[3], Pc[3];
    gmhc_push<D, Dual>(pd, Ap, gphi, Dm, vbc, vn, Pc);
    const double g = lam[0] * vn[0].d + lam[1] * vn[1].d + lam[2] * vn[2].d;
    if (q < D) ggphi[q] = g;
    else if (q < 4 * D) gDm[(q - D) / D][(q - D) % D] = g;
    else gAp[q - 4 * D] = g;
  }
  ScatterOrbit<D> so;
  so.Fbar = Fbar;
  so.pg = &pg;
  so.kc = &kc;
  so.order = 2;
  for (int l = 0; l < 3; l++) {
    so.cell[l] = cell[l];
    so.off[l] = off[l];
    so.del[l] = vb[l] * dtdx[l];
    so.gphi[l] = ggphi[l];
    for (int j = 0; j < 3; j++) so.gD1[l][j] = j < D ? gDm[l][j] * ms.inv_dx[j] : 0.0;
  }
  walk_orbit<D, double>(so.off, so.del, so, 2);
  double u1[3];
  for (int l = 0; l < 3; l++) u1[l] = off[l] + so.del[l];
  scatter_A1<D>(pg, cell, u1, gAp, Fbar, 2);
}

}  // namespace

extern "C" int pic_eval_map_vjp(pic_ctx *ctx, const double *j, const double *ybar, double tol,
                                double *H, double *jbar, int on_device) {
  if (!ctx || !j || !ybar) return PIC_EARG;
  TraceRange trace("pic_eval_map_vjp");
  if (!ctx->started) {
    ctx->err = "pic_eval_map_vjp before pic_start";
    return PIC_ESTATE;
  }
  if (ctx->rsize != 8 || ctx->opt.order != 2 || ctx->opt.refine_max != 0 ||
      ctx->opt.inner_warm_start) {
    ctx->err = "pic_eval_map_vjp: FP64, quadratic shapes, no refinement, cold inner start only";
    return PIC_EARG;
  }
  const int d = ctx->g.dim, Ng = ctx->g.Ng, nvp = node_record_len(d);
  const size_t N3 = (size_t)3 * Ng, cap = (size_t)ctx->cap;
  double tr, ta, itr, ita;
  tolerances(ctx, tol, &tr, &ta, &itr, &ita);
  const StepConst sc = make_sc(ctx, itr, ita);
  const PGeom pg = pgeom(ctx);
  // scratch: j, Jbar, H, Fbar, dual records, per particle vbar (3),
  // Phi_vbar (9) and lambda (3)
  const size_t b_vec = sizeof(double) * N3, b_F = sizeof(double) * (size_t)(d + 3) * Ng,
               b_rec = sizeof(Dual) * (size_t)Ng * nvp, b_par = sizeof(double) * 15 * cap;
  struct Scratch {
    void *p = nullptr;
    ~Scratch() {
      if (p) cudaFree(p);
    }
  } scr;
  CK(cudaMalloc(&scr.p, 3 * b_vec + b_F + b_rec + b_par));
  double *jin = (double *)scr.p, *Jb = jin + N3, *Hd = Jb + N3, *Fbar = Hd + N3;
  Dual *dnodes = (Dual *)((char *)scr.p + 3 * b_vec + b_F);
  double *vbs = (double *)((char *)scr.p + 3 * b_vec + b_F + b_rec), *jvs = vbs + 3 * cap,
         *lams = jvs + 9 * cap;
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(jin, j, b_vec, kin, ctx->st));
  CK(cudaMemcpyAsync(Jb, ybar, b_vec, kin, ctx->st));
  int e;
  if ((e = particles_step_start(ctx))) return e;
  // the primal field step and map at j (H is its projected deposit)
  if ((e = field_real_to_complex(ctx, jin, ctx->jh, 3))) return e;
  if ((e = fft_nd(ctx, ctx->jh, 3, -1))) return e;
  if ((e = field_cn_update(ctx, ctx->jh, 0))) return e;
  if ((e = field_pack_nodes(ctx, 0))) return e;
  CK(cudaMemsetAsync(ctx->Jorb, 0, b_vec, ctx->st));
  if ((e = particles_map_launch(ctx, sc, 0))) return e;
  if ((e = field_project_real(ctx, ctx->Jorb, Hd, 3))) return e;
  CK(cudaStreamSynchronize(ctx->st));
  EvalCounters cnt;
  if ((e = particles_map_finish(ctx, nullptr, nullptr, &cnt))) return e;
  if (cnt.status) {
    ctx->err = "pic_eval_map_vjp: inner particle solve failed (status bits " +
               std::to_string(cnt.status) + ")";
    return PIC_EINNER;
  }
  // Jbar = P ybar; the particles' transposes into Fbar
  if ((e = field_project_real(ctx, Jb, Jb, 3))) return e;
  CK(cudaMemsetAsync(Fbar, 0, b_F, ctx->st));
  CK(cudaMemsetAsync(ctx->cnt_dev, 0, sizeof(EvalCounters), ctx->st));
  const int64_t nrec = (int64_t)Ng * nvp;
  k_zip_rec<<<(int)((nrec + 255) / 256), 256, 0, ctx->st>>>((const double *)ctx->nodes, dnodes,
                                                            nrec);
  KCHECK();
  if (ctx->np > 0) {
    PView<double> pv;
    pv.np = ctx->np;
    pv.cap = ctx->cap;
    pv.cell = ctx->cell;
    pv.off = (const double *)ctx->off;
    pv.P = (const double *)ctx->P;
    pv.Am = (const double *)ctx->Am;
    pv.v0 = (const double *)ctx->v0;
    pv.w = ctx->w;
    pv.sp = ctx->sp;
    pv.vbar = nullptr;
    pv.Pnew = nullptr;
    pv.iters = nullptr;
    const KConst<double> kc = kconst<double>(sc, pg);
    const KConst<Dual> kcd = kconst<Dual>(sc, pg);
    const int nb = nblk(ctx->np);
    const double *nd = (const double *)ctx->nodes;
#define PIC_VJP(DD)                                                                           \
  k_vjp_phi<DD><<<nb, kPT, 0, ctx->st>>>(pv, nd, dnodes, pg, kc, kcd, vbs, jvs, ctx->cnt_dev); \
  KCHECK();                                                                                   \
  k_vjp_lambda<DD><<<nb, kPT, 0, ctx->st>>>(pv, Jb, pg, kc, kcd, vbs, jvs, lams, ctx->cnt_dev); \
  KCHECK();                                                                                   \
  k_vjp_scatter<DD><<<nb, kPT, 0, ctx->st>>>(pv, nd, vbs, lams, Fbar, pg, kc, ctx->cnt_dev);    \
  KCHECK()
    if (d == 1) {
      PIC_VJP(1);
    } else if (d == 2) {
      PIC_VJP(2);
    } else {
      PIC_VJP(3);
    }
#undef PIC_VJP
  }
  // the records' cotangents back to the trial current: forward transform,
  // the per-mode transpose of the CN step (with the inverse transform's
  // 1/Ng), unnormalised inverse transform, real part
  if ((e = field_real_to_complex(ctx, Fbar, ctx->work_h, d + 3))) return e;
  if ((e = fft_nd(ctx, ctx->work_h, d + 3, -1))) return e;
  if ((e = field_cn_adjoint(ctx, ctx->work_h, ctx->jh, 1.0 / Ng))) return e;
  if ((e = fft_nd(ctx, ctx->jh, 3, +1))) return e;
  if ((e = field_complex_to_real(ctx, ctx->jh, jin, 3, 1.0))) return e;
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (H) CK(cudaMemcpyAsync(H, Hd, b_vec, kout, ctx->st));
  if (jbar) CK(cudaMemcpyAsync(jbar, jin, b_vec, kout, ctx->st));
  CK(cudaMemcpyAsync(&cnt, ctx->cnt_dev, sizeof cnt, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (cnt.status) {
    ctx->err = "pic_eval_map_vjp: adjoint particle solve failed (status bits " +
               std::to_string(cnt.status) + ")";
    return PIC_EINNER;
  }
  return PIC_OK;
}
