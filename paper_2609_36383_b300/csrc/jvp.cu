// jvp.cu -- pic_eval_map_jvp(): one evaluation of the outer map
// H(j) = P J_orb(j) (Sec. 4.5) together with its directional derivative
// dH = H'(j) dj, the Jacobian-vector product a Newton-Krylov outer solver
// needs in place of the paper's Picard/Anderson iteration.
//
// The field step is affine in j, so its tangent is the same CN update of dj
// with the accepted state set to zero (field_cn_update_tangent).  The
// particle part is differentiated in forward mode: the particle map of
// map_device.cuh runs on dual numbers (dual.cuh) whose tangent is seeded
// from the tangent gather records (d grad phi^{1/2}, dA^{n+1}; A^n does not
// depend on j).  The inner Picard iteration then converges the orbit
// velocity and its tangent together (the tangent of the fixed point), the
// knot-split orbit integrals differentiate through their moving piece ends,
// and the deposit carries q (vbar Sbar)' / dV into a second current array.
// Both currents are projected (Eq. nyquist-projector).
#include "map_device.cuh"

#include <cstring>
#include <string>

namespace {

// dual gather records: the value from the primal records, the tangent from
// the tangent records, with the A^n slots (D .. D+2) of the tangent zero
__global__ void k_dual_records(const double *__restrict__ prim, const double *__restrict__ tan,
                               Dual *__restrict__ out, int Ng, int nvp, int d) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= (int64_t)Ng * nvp) return;
  const int slot = (int)(k % nvp);
  const bool an = slot >= d && slot < d + 3;
  out[k] = Dual(prim[k], an ? 0.0 : tan[k]);
}

// dual copies (zero tangent) of the particle inputs of the map
__global__ void k_dual_particles(int64_t np, int64_t cap, int d, const double *__restrict__ off,
                                 const double *__restrict__ P, const double *__restrict__ Am,
                                 const double *__restrict__ v0, Dual *off_d, Dual *P_d,
                                 Dual *Am_d, Dual *v0_d) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  for (int l = 0; l < d; l++) off_d[l * cap + i] = Dual(off[l * cap + i]);
  for (int c = 0; c < 3; c++) {
    P_d[c * cap + i] = Dual(P[c * cap + i]);
    Am_d[c * cap + i] = Dual(Am[c * cap + i]);
    v0_d[c * cap + i] = Dual(v0[c * cap + i]);
  }
}

struct Scratch {
  void *p = nullptr;
  ~Scratch() {
    if (p) cudaFree(p);
  }
};

}  // namespace

extern "C" int pic_eval_map_jvp(pic_ctx *ctx, const double *j, const double *dj, double tol,
                                double *H, double *dH, int on_device) {
  if (!ctx || !j || !dj) return PIC_EARG;
  if (!ctx->started) {
    ctx->err = "pic_eval_map_jvp before pic_start";
    return PIC_ESTATE;
  }
  if (ctx->rsize != 8 || ctx->opt.order != 2 || ctx->opt.refine_max != 0 ||
      ctx->opt.inner_warm_start) {
    ctx->err = "pic_eval_map_jvp: FP64, quadratic shapes, no refinement, cold inner start only";
    return PIC_EARG;
  }
  const int d = ctx->g.dim, Ng = ctx->g.Ng, nvp = node_record_len(d);
  const int64_t np = ctx->np, cap = ctx->cap;
  const size_t N3 = (size_t)3 * Ng;
  double tr, ta, itr, ita;
  tolerances(ctx, tol, &tr, &ta, &itr, &ita);
  const StepConst sc = make_sc(ctx, itr, ita);
  // scratch: zero modes, tangent records, dual records, currents, dual particles
  const size_t b_zero = sizeof(double2) * N3, b_tan = sizeof(double) * (size_t)Ng * nvp,
               b_rec = sizeof(Dual) * (size_t)Ng * nvp, b_cur = sizeof(double) * 2 * N3,
               b_par = sizeof(Dual) * (size_t)cap * (d + 15);
  Scratch scr;
  CK(cudaMalloc(&scr.p, b_zero + b_tan + b_rec + b_cur + 2 * sizeof(double) * N3 + b_par));
  char *base = (char *)scr.p;
  double2 *zero = (double2 *)base;
  double *tan_rec = (double *)(base + b_zero);
  Dual *rec = (Dual *)(base + b_zero + b_tan);
  double *Jd = (double *)(base + b_zero + b_tan + b_rec);  // [J_orb | dJ_orb]
  double *jin = Jd + 2 * N3, *djin = jin + N3;
  Dual *pd = (Dual *)(base + b_zero + b_tan + b_rec + b_cur + 2 * sizeof(double) * N3);
  Dual *off_d = pd, *P_d = pd + (size_t)d * cap, *Am_d = P_d + 3 * cap, *v0_d = Am_d + 3 * cap,
       *vb_d = v0_d + 3 * cap, *Pn_d = vb_d + 3 * cap;
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(jin, j, sizeof(double) * N3, kin, ctx->st));
  CK(cudaMemcpyAsync(djin, dj, sizeof(double) * N3, kin, ctx->st));
  CK(cudaMemsetAsync(zero, 0, b_zero, ctx->st));
  CK(cudaMemsetAsync(Jd, 0, b_cur, ctx->st));
  CK(cudaMemsetAsync(ctx->cnt_dev, 0, sizeof(EvalCounters), ctx->st));
  int e;
  if ((e = particles_step_start(ctx))) return e;
  // tangent field step, then its gather records (kept apart)
  if ((e = field_real_to_complex(ctx, djin, ctx->jh, 3))) return e;
  if ((e = fft_nd(ctx, ctx->jh, 3, -1))) return e;
  if ((e = field_cn_update_tangent(ctx, ctx->jh, zero))) return e;
  if ((e = field_pack_nodes(ctx, 0))) return e;
  CK(cudaMemcpyAsync(tan_rec, ctx->nodes, b_tan, cudaMemcpyDeviceToDevice, ctx->st));
  // primal field step (overwrites the candidate n+1 buffers and A1_real)
  if ((e = field_real_to_complex(ctx, jin, ctx->jh, 3))) return e;
  if ((e = fft_nd(ctx, ctx->jh, 3, -1))) return e;
  if ((e = field_cn_update(ctx, ctx->jh, 0))) return e;
  if ((e = field_pack_nodes(ctx, 0))) return e;
  {
    const int64_t n = (int64_t)Ng * nvp;
    k_dual_records<<<(int)((n + 255) / 256), 256, 0, ctx->st>>>((const double *)ctx->nodes,
                                                                 tan_rec, rec, Ng, nvp, d);
    KCHECK();
  }
  if (np > 0) {
    k_dual_particles<<<nblk(np), kPT, 0, ctx->st>>>(np, cap, d, (const double *)ctx->off,
                                                    (const double *)ctx->P,
                                                    (const double *)ctx->Am,
                                                    (const double *)ctx->v0, off_d, P_d, Am_d,
                                                    v0_d);
    KCHECK();
    PView<Dual> pv;
    pv.np = np;
    pv.cap = cap;
    pv.cell = ctx->cell;
    pv.off = off_d;
    pv.P = P_d;
    pv.Am = Am_d;
    pv.v0 = v0_d;
    pv.w = ctx->w;
    pv.sp = ctx->sp;
    pv.vbar = vb_d;
    pv.Pnew = Pn_d;
    pv.iters = ctx->iters;
    const PGeom pg = pgeom(ctx);
    const KConst<Dual> kc = kconst<Dual>(sc, pg);
    if (d == 1)
      k_map<1, Dual, false, false><<<nblk(np), kPT, 0, ctx->st>>>(pv, rec, rec, Jd, pg, kc,
                                                                  ctx->cnt_dev, ctx->psum);
    else if (d == 2)
      k_map<2, Dual, false, false><<<nblk(np), kPT, 0, ctx->st>>>(pv, rec, rec, Jd, pg, kc,
                                                                  ctx->cnt_dev, ctx->psum);
    else
      k_map<3, Dual, false, false><<<nblk(np), kPT, 0, ctx->st>>>(pv, rec, rec, Jd, pg, kc,
                                                                  ctx->cnt_dev, ctx->psum);
    KCHECK();
  }
  // H = P J_orb and dH = P dJ_orb
  if ((e = field_project_real(ctx, Jd, Jd, 3))) return e;
  if ((e = field_project_real(ctx, Jd + N3, Jd + N3, 3))) return e;
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (H) CK(cudaMemcpyAsync(H, Jd, sizeof(double) * N3, kout, ctx->st));
  if (dH) CK(cudaMemcpyAsync(dH, Jd + N3, sizeof(double) * N3, kout, ctx->st));
  EvalCounters cnt;
  CK(cudaMemcpyAsync(&cnt, ctx->cnt_dev, sizeof cnt, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (cnt.status) {
    ctx->err = "pic_eval_map_jvp: inner particle solve failed (status bits " +
               std::to_string(cnt.status) + ")";
    return PIC_EINNER;
  }
  return PIC_OK;
}
