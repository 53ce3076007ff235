// step_adjoint.cu -- pic_step_vjp(): the adjoint (reverse mode) of one
// implicit step, Sbar^n = (dS^{n+1}/dS^n)^T Sbar^{n+1}, for gradients with
// respect to many parameters of the state at once.  The paper differentiates
// nothing; this transposes the step of Sec. 4.5 / Algorithm 1 that
// pic_tangent_* differentiates forward.
//
// A step maps the state S = (x, P; phi, psi, A, U, rho) to
// S' = G(j*, S), where the converged current solves j* = H(j*, S) and G
// commits the particles (x' = x + dt vbar, P' = P^{n+1} of the push) and the
// field step.  By implicit differentiation
//     Sbar = G_S^T Sbar' + H_S^T lambda,  (I - H_j^T) lambda = G_j^T Sbar'.
// Both terms are one "generalised VJP" of a map evaluation at (j*, S): given
// cotangents on the committed particles (xbar', Pbar'), on the next field
// state, and on the deposited current (Jbar = P lambda, the projector being
// symmetric), it returns the cotangents of j and of S.  Per particle the
// inner fixed point vbar = Phi(vbar; x, P, A^-, records) transposes as in
// the adjoint of a map evaluation (adjoint.cu): mu solves
// (I - Phi_vbar^T) mu = dt xbar' + (dP'/dvbar)^T Pbar' + grad_vbar s, with s
// the deposit's scalar q vbar . G(Jbar)/dV, and the push's transpose on
// (mu, Pbar') gives the cotangents of x (dual sweeps on the in-cell offset,
// through the orbit gather, A^- = A^n(x) and the deposit's weights), of P
// (dual pushes) and of the node records [grad phi^{1/2}, A^n, A^{n+1}]
// (scattered with the gather's orbit weights; A^- scattered at the start
// point).  The field step is linear; its transpose is k_cn_state_adjoint
// between forward and inverse transforms.  The outer equation for lambda is
// solved by restarted GMRES on the j-part of the generalised VJP.
//
// The call recomputes the step (orbits are recomputed, nothing is stored by
// the forward run): it snapshots the state on the device, runs pic_step for
// j*, copies the snapshot back, and differentiates at (j*, S^n).  The
// context's state is unchanged on return.
#include "adjoint_device.cuh"
#include "trace.cuh"

#include <cmath>
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

namespace {

constexpr int kAdjKrylov = 20;
constexpr int kAdjRestarts = 6;
// A restart that gains less than a factor 2 below kAdjNoiseFloor (relative)
// has reached the accuracy the operator's rounding allows (its applications
// sum with atomics and converge inner solves to a tolerance): accepted.
constexpr double kAdjNoiseFloor = 1e-9;

// dA^n_c / d off_l at the particle's start (quadratic shapes): the gradient
// of point_interp_T in node units
template <int D>
__device__ void point_grad(const PGeom &pg, const int cell[3], const double off[3],
                           const double *__restrict__ A, double gA[3][3]) {
  int base[3] = {0, 0, 0};
  double S[3][3], dS[3][3];
  for (int l = 0; l < 3; l++)
    for (int o = 0; o < 3; o++) {
      S[l][o] = 0.0;
      dS[l][o] = 0.0;
    }
  for (int l = 0; l < D; l++) {
    base[l] = (int)floor(off[l] + 0.5);
    qspline<double>(off[l] - double(base[l]), S[l], dS[l]);
  }
  for (int c = 0; c < 3; c++)
    for (int l = 0; l < 3; l++) gA[c][l] = 0.0;
  const NodeRows<D> nr(pg, cell, base);
  const size_t Ng = (size_t)pg.Ng;
  for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
    for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
      for (int ox = 0; ox < 3; ox++) {
        const int g = nr.at(ox, oy, oz);
        const int idx[3] = {ox, oy, oz};
        for (int l = 0; l < D; l++) {
          double w = 1.0;
          for (int m = 0; m < D; m++) w *= m == l ? dS[m][idx[m]] : S[m][idx[m]];
          for (int c = 0; c < 3; c++) gA[c][l] += w * A[c * Ng + g];
        }
      }
}

// transpose of the point interpolation of a 3-component mesh field at u
// (node units relative to the cell): g scattered with the point weights
template <int D>
__device__ void scatter_point(const PGeom &pg, const int cell[3], const double u[3],
                              const double g3[3], double *Fslot) {
  int base[3] = {0, 0, 0};
  double Sw[3][3];
  for (int l = 0; l < D; l++) {
    base[l] = (int)floor(u[l] + 0.5);
    spline_val<double>(2, u[l] - double(base[l]), Sw[l]);
  }
  const NodeRows<D> nr(pg, cell, base);
  const size_t Ng = (size_t)pg.Ng;
  for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
    for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
      for (int ox = 0; ox < 3; ox++) {
        const int g = nr.at(ox, oy, oz);
        const double w = Sw[0][ox] * (D > 1 ? Sw[1][oy] : 1.0) * (D > 2 ? Sw[2][oz] : 1.0);
        for (int c = 0; c < 3; c++) atomicAdd(Fslot + c * Ng + g, w * g3[c]);
      }
}

// The transpose of GatherOrbit with respect to every record it reads:
// grad phi^{1/2} (weights Sbar), A^{n+1} (weights W1) and, when An is set,
// A^n (weights Wd - W1, since D_i A = sum A^n Wd + (A^{n+1} - A^n) W1).
// Fbar = [grad phi (D), A^{n+1} (3), A^n (3)] x Ng.
template <int D>
struct ScatterOrbitFull {
  double *__restrict__ Fbar;
  const PGeom *pg;
  const KConst<double> *kc;
  int cell[3];
  double off[3], del[3];
  double gphi[3], gD[3][3];  // gD: cotangent of D_i A with columns per node unit
  bool An;
  __device__ __forceinline__ void put(size_t Ng, int g, double Sb, const double Wd[3],
                                      const double W1[3]) {
    for (int c = 0; c < D; c++) atomicAdd(Fbar + c * Ng + g, Sb * gphi[c]);
    for (int c = 0; c < 3; c++) {
      double v1 = 0.0, v0 = 0.0;
      for (int j = 0; j < D; j++) {
        v1 += W1[j] * gD[c][j];
        v0 += (Wd[j] - W1[j]) * gD[c][j];
      }
      atomicAdd(Fbar + (D + c) * Ng + g, v1);
      if (An) atomicAdd(Fbar + (D + 3 + c) * Ng + g, v0);
    }
  }
  __device__ __forceinline__ void operator()(const int base[3], double sa, double sb) {
    const NodeRows<D> nr(*pg, cell, base);
    const size_t Ng = (size_t)pg->Ng;
    if (D == 3) {
#pragma unroll 1
      for (int oz = 0; oz < 3; oz++) {
        PieceAcc<2, double> pa;
        double Wz[9], W1z[9];
        accumulate_slab<double, true>(*kc, off, del, base, sa, sb, oz, pa, Wz, W1z, 2);
        for (int oy = 0; oy < 3; oy++)
          for (int ox = 0; ox < 3; ox++) {
            const int k = ox + 3 * oy;
            const double Wd[3] = {pa.Wd[0][k], pa.Wd[1][k], Wz[k]};
            const double W1[3] = {pa.W1[0][k], pa.W1[1][k], W1z[k]};
            put(Ng, nr.at(ox, oy, oz), pa.Sb[k], Wd, W1);
          }
      }
      return;
    }
    PieceAcc<D, double> pa;
    accumulate_piece<D, double, true>(*kc, off, del, base, sa, sb, pa, 2);
    for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
      for (int ox = 0; ox < 3; ox++) {
        const int k = ox + 3 * oy;
        double Wd[3] = {0.0, 0.0, 0.0}, W1[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < D; j++) {
          Wd[j] = pa.Wd[j][k];
          W1[j] = pa.W1[j][k];
        }
        put(Ng, nr.at(ox, oy, 0), pa.Sb[k], Wd, W1);
      }
  }
};

// Pass A, one thread per particle: converge vbar as the map does (cold
// start), then from three dual sweeps with the velocity seeded the columns
// of dvn/dvbar (Phi_vbar, 9 x cap) and dP^{n+1}/dvbar (9 x cap).
template <int D>
__global__ void k_sadj_jac(PView<double> pv, const double *__restrict__ nodes,
                           const Dual *__restrict__ dnodes, PGeom pg, KConst<double> kc,
                           KConst<Dual> kcd, double *__restrict__ vb_out,
                           double *__restrict__ jv_out, double *__restrict__ jp_out,
                           EvalCounters *__restrict__ cnt) {
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
    for (int c = 0; c < 3; c++) {
      jv_out[(size_t)(c * 3 + e) * pv.cap + i] = vn[c].d;
      jp_out[(size_t)(c * 3 + e) * pv.cap + i] = Pc[c].d;
    }
  }
  for (int c = 0; c < 3; c++) vb_out[(size_t)c * pv.cap + i] = vb[c];
}

// Pass B: the particle's cotangent mu of the inner fixed point from
// (I - Phi_vbar^T) mu = dt xbar' + (dP^{n+1}/dvbar)^T Pbar' + grad_vbar s,
// with s = q vbar . G(Jbar; vbar) / dV the deposit's scalar (three orbit
// gathers on dual numbers).  Any of xb1, Pb1, Jbar may be null (zero).
template <int D>
__global__ void k_sadj_mu(PView<double> pv, const double *__restrict__ Jbar, PGeom pg,
                          KConst<double> kc, KConst<Dual> kcd, const double *__restrict__ vb_in,
                          const double *__restrict__ jv_in, const double *__restrict__ jp_in,
                          const double *__restrict__ xb1, const double *__restrict__ Pb1,
                          double *__restrict__ mu_out, EvalCounters *__restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np || cnt->status) return;
  const int64_t cap = pv.cap;
  const MapScale<double> ms = {{kc.inv_dx[0], kc.inv_dx[1], kc.inv_dx[2]}, kc.inv_dV};
  PushConst<double> pc;
  int cell[3];
  double off[3], dtdx[3], vb[3], Jv[3][3], b[3] = {0.0, 0.0, 0.0};
  vjp_particle<D>(pv, i, kc, ms, pc, cell, off, dtdx);
  for (int c = 0; c < 3; c++) {
    vb[c] = vb_in[(size_t)c * cap + i];
    for (int e = 0; e < 3; e++) Jv[c][e] = jv_in[(size_t)(c * 3 + e) * cap + i];
  }
  if (Pb1)
    for (int e = 0; e < 3; e++)
      for (int c = 0; c < 3; c++) b[e] += jp_in[(size_t)(c * 3 + e) * cap + i] * Pb1[c * cap + i];
  if (xb1)
    for (int l = 0; l < D; l++) b[l] += kc.dt * xb1[l * cap + i];
  if (Jbar) {
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
      b[e] += sv.d;
    }
  }
  double mu[3];
  if (!solve_adjoint3(Jv, b, mu)) {
    atomicOr(&cnt->status, PIC_ST_NONFINITE);
    return;
  }
  for (int c = 0; c < 3; c++) mu_out[(size_t)c * cap + i] = mu[c];
}

// One push on dual numbers at the converged orbit (gathered quantities and
// velocity constant), with the push constants pd carrying the seed; returns
// mu . dvn + Pbar' . dP^{n+1}.
template <int D>
__device__ double push_dot(const PushConst<Dual> &pd, const double gphi0[3], const double Dm0[3][3],
                           const double Ap0[3], const double vb[3], const double mu[3],
                           const double Pb[3]) {
  Dual gphi[3], Dm[3][3], Ap[3], vbc[3], vn[3], Pc[3];
  for (int c = 0; c < 3; c++) {
    gphi[c] = Dual(gphi0[c]);
    Ap[c] = Dual(Ap0[c]);
    vbc[c] = Dual(vb[c]);
    for (int j = 0; j < 3; j++) Dm[c][j] = Dual(Dm0[c][j]);
  }
  gmhc_push<D, Dual>(pd, Ap, gphi, Dm, vbc, vn, Pc);
  double s = 0.0;
  for (int c = 0; c < 3; c++) s += mu[c] * vn[c].d + Pb[c] * Pc[c].d;
  return s;
}

// The particle's primal at the converged orbit, shared by the passes below:
// push constants, position, vbar, mu, Pbar', and the gathered quantities.
template <int D>
struct SadjParticle {
  PushConst<double> pc;
  int cell[3];
  double off[3], dtdx[3], vb[3], mu[3], Pb[3];
  double gphi0[3], Dm0[3][3], Ap0[3];
  // false when the orbit is too long for the walk (flagged by the first pass,
  // after which no later pass runs): the gathered values are then not set
  __device__ bool load(const PView<double> &pv, int64_t i, const double *__restrict__ nodes,
                       const PGeom &pg, const KConst<double> &kc, const MapScale<double> &ms,
                       const double *__restrict__ vb_in, const double *__restrict__ mu_in,
                       const double *__restrict__ Pb1) {
    const int64_t cap = pv.cap;
    vjp_particle<D>(pv, i, kc, ms, pc, cell, off, dtdx);
    for (int c = 0; c < 3; c++) {
      vb[c] = vb_in[(size_t)c * cap + i];
      mu[c] = mu_in[(size_t)c * cap + i];
      Pb[c] = Pb1 ? Pb1[c * cap + i] : 0.0;
    }
    int np2 = 0;
    return orbit_gather<D, double, false>(cell, off, dtdx, 0.0, 1.0, nodes, pg, kc, ms, vb, gphi0,
                                          Dm0, Ap0, np2, 2);
  }
};

// Pass C1: the push's transpose on (mu, Pbar') over the gathered quantities
// (one dual push per quantity), scattered to the records Fbar = [grad phi
// (D), A^{n+1} (3), A^n (3)] with the gather's orbit weights; the A^n part
// only with want_state.
template <int D>
__global__ void k_sadj_records(PView<double> pv, const double *__restrict__ nodes, PGeom pg,
                               KConst<double> kc, const double *__restrict__ vb_in,
                               const double *__restrict__ mu_in, const double *__restrict__ Pb1,
                               int want_state, double *__restrict__ Fbar,
                               const EvalCounters *__restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np || cnt->status) return;
  const MapScale<double> ms = {{kc.inv_dx[0], kc.inv_dx[1], kc.inv_dx[2]}, kc.inv_dV};
  SadjParticle<D> sp;
  if (!sp.load(pv, i, nodes, pg, kc, ms, vb_in, mu_in, Pb1)) return;
  const PushConst<Dual> pd0 = dual_push_const(sp.pc);
  double ggphi[3] = {0.0, 0.0, 0.0}, gDm[3][3] = {{0.0}}, gAp[3] = {0.0, 0.0, 0.0};
  const int nin = D + 3 * D + 3;  // grad phi (D), D_i A (3 x D), A^{n+1} (3)
  for (int q = 0; q < nin; q++) {
    Dual gphi[3], Dm[3][3], Ap[3], vbc[3], vn[3], Pc[3];
    for (int c = 0; c < 3; c++) {
      gphi[c] = Dual(sp.gphi0[c]);
      Ap[c] = Dual(sp.Ap0[c]);
      vbc[c] = Dual(sp.vb[c]);
      for (int j = 0; j < 3; j++) Dm[c][j] = Dual(sp.Dm0[c][j]);
    }
    if (q < D) gphi[q].d = 1.0;
    else if (q < 4 * D) Dm[(q - D) / D][(q - D) % D].d = 1.0;
    else Ap[q - 4 * D].d = 1.0;
    gmhc_push<D, Dual>(pd0, Ap, gphi, Dm, vbc, vn, Pc);
    double g = 0.0;
    for (int c = 0; c < 3; c++) g += sp.mu[c] * vn[c].d + sp.Pb[c] * Pc[c].d;
    if (q < D) ggphi[q] = g;
    else if (q < 4 * D) gDm[(q - D) / D][(q - D) % D] = g;
    else gAp[q - 4 * D] = g;
  }
  ScatterOrbitFull<D> so;
  so.Fbar = Fbar;
  so.pg = &pg;
  so.kc = &kc;
  so.An = want_state != 0;
  for (int l = 0; l < 3; l++) {
    so.cell[l] = sp.cell[l];
    so.off[l] = sp.off[l];
    so.del[l] = sp.vb[l] * sp.dtdx[l];
    so.gphi[l] = ggphi[l];
    for (int j = 0; j < 3; j++) so.gD[l][j] = j < D ? gDm[l][j] * ms.inv_dx[j] : 0.0;
  }
  walk_orbit<D, double>(so.off, so.del, so, 2);
  double u1[3];
  for (int l = 0; l < 3; l++) u1[l] = sp.off[l] + so.del[l];
  scatter_point<D>(pg, sp.cell, u1, gAp, Fbar + (size_t)D * pg.Ng);
}

// Pass C2: the cotangents of the particle's P (dual pushes: P^n and
// p^n = P^n - q A^- move together, and gamma_n with p^n) into Pb0, and of
// A^- = A^n(x) (dual pushes), scattered at the start point into the A^n slot
// of Fbar.
template <int D>
__global__ void k_sadj_momentum(PView<double> pv, const double *__restrict__ nodes, PGeom pg,
                                KConst<double> kc, const double *__restrict__ vb_in,
                                const double *__restrict__ mu_in,
                                const double *__restrict__ Pb1, double *__restrict__ Fbar,
                                double *__restrict__ Pb0, const EvalCounters *__restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np || cnt->status) return;
  const MapScale<double> ms = {{kc.inv_dx[0], kc.inv_dx[1], kc.inv_dx[2]}, kc.inv_dV};
  SadjParticle<D> sp;
  if (!sp.load(pv, i, nodes, pg, kc, ms, vb_in, mu_in, Pb1)) return;
  const PushConst<double> &pc = sp.pc;
  const PushConst<Dual> pd0 = dual_push_const(pc);
  const double ik2 = pc.inv_mk * pc.inv_mk;
  for (int e = 0; e < 3; e++) {
    PushConst<Dual> pd = pd0;
    pd.Pn[e].d = 1.0;
    pd.pn[e].d = 1.0;
    pd.gamma_n.d = pc.pn[e] * ik2 / pc.gamma_n;
    Pb0[e * pv.cap + i] = push_dot<D>(pd, sp.gphi0, sp.Dm0, sp.Ap0, sp.vb, sp.mu, sp.Pb);
  }
  double gAm[3];
  for (int e = 0; e < 3; e++) {
    PushConst<Dual> pd = pd0;
    pd.Am[e].d = 1.0;
    pd.pn[e].d = -pc.q;
    pd.gamma_n.d = -pc.q * pc.pn[e] * ik2 / pc.gamma_n;
    gAm[e] = push_dot<D>(pd, sp.gphi0, sp.Dm0, sp.Ap0, sp.vb, sp.mu, sp.Pb);
  }
  scatter_point<D>(pg, sp.cell, sp.off, gAm, Fbar + (size_t)(D + 3) * pg.Ng);
}

// Pass C3: the cotangent of x: one dual sweep per active dimension with the
// in-cell offset seeded, through the orbit gather (and A^+ at the orbit's
// end), A^- = A^n(x) in the push constants and the deposit's weights, plus
// the identity of x' = x + dt vbar; into xb0 (D x cap).
template <int D>
__global__ void k_sadj_position(PView<double> pv, const double *__restrict__ nodes,
                                const Dual *__restrict__ dnodes, const double *__restrict__ A_n,
                                const double *__restrict__ Jbar, PGeom pg, KConst<double> kc,
                                KConst<Dual> kcd, const double *__restrict__ vb_in,
                                const double *__restrict__ mu_in, const double *__restrict__ xb1,
                                const double *__restrict__ Pb1, double *__restrict__ xb0,
                                const EvalCounters *__restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np || cnt->status) return;
  const int64_t cap = pv.cap;
  const MapScale<double> ms = {{kc.inv_dx[0], kc.inv_dx[1], kc.inv_dx[2]}, kc.inv_dV};
  const MapScale<Dual> msd = {{kcd.inv_dx[0], kcd.inv_dx[1], kcd.inv_dx[2]}, kcd.inv_dV};
  PushConst<double> pc;
  int cell[3];
  double off[3], dtdx[3], vb[3], mu[3], Pb[3];
  vjp_particle<D>(pv, i, kc, ms, pc, cell, off, dtdx);
  for (int c = 0; c < 3; c++) {
    vb[c] = vb_in[(size_t)c * cap + i];
    mu[c] = mu_in[(size_t)c * cap + i];
    Pb[c] = Pb1 ? Pb1[c * cap + i] : 0.0;
  }
  const PushConst<Dual> pd0 = dual_push_const(pc);
  const double ik2 = pc.inv_mk * pc.inv_mk;
  double gA[3][3];
  point_grad<D>(pg, cell, off, A_n, gA);
  Dual dtdxd[3], vbd[3];
  for (int l = 0; l < 3; l++) {
    dtdxd[l] = Dual(dtdx[l]);
    vbd[l] = Dual(vb[l]);
  }
  const Dual qdv(pc.q * ms.inv_dV);
  for (int l = 0; l < D; l++) {
    PushConst<Dual> pd = pd0;
    double dg = 0.0;
    for (int c = 0; c < 3; c++) {
      pd.Am[c].d = gA[c][l];
      pd.pn[c].d = -pc.q * gA[c][l];
      dg += pc.pn[c] * (-pc.q * gA[c][l]);
    }
    pd.gamma_n.d = dg * ik2 / pc.gamma_n;
    Dual offd[3];
    for (int m = 0; m < 3; m++) offd[m] = Dual(off[m], m == l ? 1.0 : 0.0);
    Dual gphi[3], Dm[3][3], Ap[3], vn[3], Pc[3];
    int np_ = 0;
    if (!orbit_gather<D, Dual, false>(cell, offd, dtdxd, Dual(0.0), Dual(1.0), dnodes, pg, kcd,
                                      msd, vbd, gphi, Dm, Ap, np_, 2))
      return;  // flagged by the first pass, as in SadjParticle::load
    gmhc_push<D, Dual>(pd, Ap, gphi, Dm, vbd, vn, Pc);
    double val = 0.0;
    for (int c = 0; c < 3; c++) val += mu[c] * vn[c].d + Pb[c] * Pc[c].d;
    if (Jbar) {
      OrbitDot<D, Dual> od;
      od.F = Jbar;
      od.pg = &pg;
      od.kc = &kcd;
      od.order = 2;
      for (int m = 0; m < 3; m++) {
        od.cell[m] = cell[m];
        od.off[m] = offd[m];
        od.del[m] = vbd[m] * dtdxd[m];
        od.G[m] = Dual(0.0);
      }
      walk_orbit<D, Dual>(od.off, od.del, od, 2);
      Dual sv(0.0);
      for (int c = 0; c < 3; c++) sv += qdv * vbd[c] * od.G[c];
      val += sv.d;
    }
    xb0[l * cap + i] = val * ms.inv_dx[l] + (xb1 ? xb1[l * cap + i] : 0.0);
  }
}

// per-particle rows between load order (caller) and slot order (storage)
__global__ void k_rows_to_slot(const double *__restrict__ src, double *__restrict__ dst,
                               const int64_t *__restrict__ id, int64_t np, int64_t cap,
                               int nrows) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int64_t k = id[i];
  for (int r = 0; r < nrows; r++) dst[r * cap + i] = src[r * np + k];
}

__global__ void k_rows_to_load(const double *__restrict__ src, double *__restrict__ dst,
                               const int64_t *__restrict__ id, int64_t np, int64_t cap,
                               int nrows) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int64_t k = id[i];
  for (int r = 0; r < nrows; r++) dst[r * np + k] = src[r * cap + i];
}

inline unsigned grid_of(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

namespace {

// Euclidean norm of a 3 Ng mesh vector
double vnorm(pic_ctx *ctx, const double *a, int *err) {
  const double *pa[1] = {a};
  double v = 0.0;
  *err = dots(ctx, pa, pa, 1, &v);
  return std::sqrt(v);
}

// Restarted GMRES(kAdjKrylov) for A x = b on 3 Ng mesh vectors, A given as
// an operator; Arnoldi with two passes of classical Gram-Schmidt, Givens
// rotations on the host.  x starts at zero.  Converged when the true
// residual is below rtol times max(|b|, |x|).
int gmres_solve(pic_ctx *ctx, const std::function<int(const double *, double *)> &op,
                const double *b, double *x, double *ws, double rtol, int *iters) {
  const size_t N = (size_t)3 * ctx->g.Ng;
  const int m = kAdjKrylov;
  double *V = ws, *w = V + (size_t)(m + 1) * N;
  int e;
  *iters = 0;
  CK(cudaMemsetAsync(x, 0, sizeof(double) * N, ctx->st));
  const double bn = vnorm(ctx, b, &e);
  if (e) return e;
  if (!std::isfinite(bn)) {
    ctx->err = "pic_step_vjp: non-finite right-hand side";
    return PIC_EOUTER;
  }
  if (bn == 0.0) return PIC_OK;
  CK(cudaMemcpyAsync(V, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, ctx->st));
  double beta = bn, ref = bn, beta_prev = bn;
  std::string hist;
  for (int restart = 0; restart < kAdjRestarts; restart++) {
    if ((e = lincomb(ctx, V, V, 1.0 / beta, V, 0.0, N))) return e;
    std::vector<double> H((m + 1) * m, 0.0), g(m + 1, 0.0), cs(m, 0.0), sn(m, 0.0);
    g[0] = beta;
    int kk = 0;
    for (int k = 0; k < m; k++) {
      double *Vk = V + (size_t)k * N, *Vn = V + (size_t)(k + 1) * N;
      if ((e = op(Vk, w))) return e;
      (*iters)++;
      for (int pass = 0; pass < 2; pass++) {
        const double *pa[kAdjKrylov + 1], *pb[kAdjKrylov + 1];
        double h[kAdjKrylov + 1];
        for (int i = 0; i <= k; i++) {
          pa[i] = V + (size_t)i * N;
          pb[i] = w;
        }
        if ((e = dots(ctx, pa, pb, k + 1, h))) return e;
        for (int i = 0; i <= k; i++) {
          H[i * m + k] += h[i];
          if ((e = lincomb(ctx, w, w, 1.0, pa[i], -h[i], N))) return e;
        }
      }
      const double hn = vnorm(ctx, w, &e);
      if (e) return e;
      if (!std::isfinite(hn)) {
        ctx->err = "pic_step_vjp: non-finite Krylov vector";
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
      if (hn > 0.0 && (e = lincomb(ctx, Vn, w, 1.0 / hn, w, 0.0, N))) return e;
      if (std::fabs(g[k + 1]) <= 0.5 * rtol * ref || hn == 0.0) break;
    }
    std::vector<double> y(kk, 0.0);
    for (int i = kk - 1; i >= 0; i--) {
      double s = g[i];
      for (int q = i + 1; q < kk; q++) s -= H[i * m + q] * y[q];
      y[i] = H[i * m + i] != 0.0 ? s / H[i * m + i] : 0.0;
    }
    for (int i = 0; i < kk; i++)
      if ((e = lincomb(ctx, x, x, 1.0, V + (size_t)i * N, y[i], N))) return e;
    // true residual b - A x into V_0
    if ((e = op(x, w))) return e;
    if ((e = lincomb(ctx, V, b, 1.0, w, -1.0, N))) return e;
    beta = vnorm(ctx, V, &e);
    if (e) return e;
    ref = std::fmax(bn, vnorm(ctx, x, &e));
    if (e) return e;
    char buf[32];
    std::snprintf(buf, sizeof buf, "%s%.3e", hist.empty() ? "" : ", ", beta / ref);
    hist += buf;
    if (!std::isfinite(beta)) break;
    if (beta <= rtol * ref) return PIC_OK;
    if (beta > 0.5 * beta_prev && beta <= kAdjNoiseFloor * ref) return PIC_OK;
    beta_prev = beta;
  }
  ctx->err = "pic_step_vjp: GMRES did not reach the tolerance (relative residuals " + hist + ")";
  return PIC_EOUTER;
}

}  // namespace

extern "C" int pic_step_vjp(pic_ctx *ctx, double tol, const double *xbar1, const double *Pbar1,
                            const double *fbar1, double *xbar0, double *Pbar0, double *fbar0,
                            int *gmres_iters, int on_device) {
  if (!ctx) return PIC_EARG;
  TraceRange trace("pic_step_vjp");
  if (!ctx->started) {
    ctx->err = "pic_step_vjp before pic_start";
    return PIC_ESTATE;
  }
  if (ctx->rsize != 8 || ctx->opt.order != 2 || ctx->opt.refine_max != 0 ||
      ctx->opt.inner_warm_start) {
    ctx->err = "pic_step_vjp: FP64, quadratic shapes, no refinement, cold inner start only";
    return PIC_EARG;
  }
  if (gmres_iters) *gmres_iters = 0;
  const int d = ctx->g.dim, Ng = ctx->g.Ng, nvp = node_record_len(d);
  const size_t N3 = (size_t)3 * Ng;
  int e;
  // 1. the step itself, for j*; a device snapshot of the state brings S^n back
  struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
      if (p) cudaFree(p);
    }
  } snap;
  CK(cudaMalloc(&snap.p, state_snapshot_bytes(ctx)));
  if ((e = state_snapshot(ctx, snap.p))) return e;
  const int64_t np = ctx->np;
  const size_t cap = (size_t)ctx->cap;
  // scratch, before the step, so that nothing after the step can fail
  // before the snapshot is restored but a copy (a step keeps np and cap)
  const size_t n_mesh = (size_t)(d + 6) * Ng  // Fbar
                        + 9 * (size_t)Ng      // next-state cotangents (real)
                        + 9 * (size_t)Ng      // current-state cotangents (real)
                        + 5 * N3              // j*, jbar, Jbar, rhs, lambda
                        + (size_t)(kAdjKrylov + 2) * N3;  // GMRES basis + w
  const size_t n_spec = (size_t)(9 + 9 + (d + 3) + 12) * Ng;  // Ybar, zeros, Rbar, out
  const size_t n_part = 3 + 9 + 9 + 3 + 3 + 3 + 3 + 3 + 3;  // vb jv jp mu xb1 Pb1 xb0 Pb0 tmp
  struct Scratch {
    void *p = nullptr;
    ~Scratch() {
      if (p) cudaFree(p);
    }
  } scr;
  const size_t b_mesh = sizeof(double) * n_mesh, b_spec = sizeof(double2) * n_spec,
               b_rec = sizeof(Dual) * (size_t)Ng * nvp,
               b_part = sizeof(double) * n_part * (cap > 0 ? cap : 1);
  CK(cudaMalloc(&scr.p, b_mesh + b_spec + b_rec + b_part));
  double *Fbar = (double *)scr.p;
  double *f1 = Fbar + (size_t)(d + 6) * Ng, *f0 = f1 + 9 * (size_t)Ng;
  double *jstar = f0 + 9 * (size_t)Ng, *jbar = jstar + N3, *Jb = jbar + N3, *rhs = Jb + N3,
         *lam = rhs + N3, *gws = lam + N3;
  double2 *Ys = (double2 *)((char *)scr.p + b_mesh), *Zs = Ys + 9 * (size_t)Ng,
          *Rs = Zs + 9 * (size_t)Ng, *Os = Rs + (size_t)(d + 3) * Ng;
  Dual *dnodes = (Dual *)((char *)scr.p + b_mesh + b_spec);
  double *vbs = (double *)((char *)scr.p + b_mesh + b_spec + b_rec);
  double *jvs = vbs + 3 * cap, *jps = jvs + 9 * cap, *mus = jps + 9 * cap, *xb1s = mus + 3 * cap,
         *Pb1s = xb1s + 3 * cap, *xb0s = Pb1s + 3 * cap, *Pb0s = xb0s + 3 * cap,
         *ptmp = Pb0s + 3 * cap;  // 3 x np rows in load order
  const long long steps0 = ctx->steps_done;
  const int sort0 = ctx->opt.sort_every;
  const double E00 = ctx->E0;
  pic_report rep;
  const int st_step = pic_step(ctx, tol, &rep);
  if (st_step != PIC_OK) return st_step;  // a failed step leaves S^n in place
  // S^n goes back in place whatever the copy of j* returns; the copy's
  // status is checked only after the restore
  const cudaError_t ce_j =
      cudaMemcpyAsync(jstar, ctx->J_acc, sizeof(double) * N3, cudaMemcpyDeviceToDevice, ctx->st);
  if ((e = state_restore(ctx, snap.p, np, steps0, sort0, E00))) return e;
  CK(ce_j);
  CK(cudaStreamSynchronize(ctx->st));
  // 2. the map evaluation at (j*, S^n): records, then vbar and its Jacobians
  const StepConst sc = [&] {
    double tr, ta, itr, ita;
    tolerances(ctx, tol, &tr, &ta, &itr, &ita);
    return make_sc(ctx, itr, ita);
  }();
  const PGeom pg = pgeom(ctx);
  if ((e = particles_step_start(ctx))) return e;
  if ((e = field_real_to_complex(ctx, jstar, ctx->jh, 3))) return e;
  if ((e = fft_nd(ctx, ctx->jh, 3, -1))) return e;
  if ((e = field_cn_update(ctx, ctx->jh, 0))) return e;
  if ((e = field_pack_nodes(ctx, 0))) return e;
  const int64_t nrec = (int64_t)Ng * nvp;
  k_zip_rec<<<grid_of(nrec), 256, 0, ctx->st>>>((const double *)ctx->nodes, dnodes, nrec);
  KCHECK();
  CK(cudaMemsetAsync(ctx->cnt_dev, 0, sizeof(EvalCounters), ctx->st));
  PView<double> pv;
  pv.np = np;
  pv.cap = (int64_t)cap;
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
  const double *nd = (const double *)ctx->nodes;
  const unsigned nb = (unsigned)nblk(np > 0 ? np : 1);
  if (np > 0) {
    if (d == 1) k_sadj_jac<1><<<nb, kPT, 0, ctx->st>>>(pv, nd, dnodes, pg, kc, kcd, vbs, jvs, jps, ctx->cnt_dev);
    else if (d == 2) k_sadj_jac<2><<<nb, kPT, 0, ctx->st>>>(pv, nd, dnodes, pg, kc, kcd, vbs, jvs, jps, ctx->cnt_dev);
    else k_sadj_jac<3><<<nb, kPT, 0, ctx->st>>>(pv, nd, dnodes, pg, kc, kcd, vbs, jvs, jps, ctx->cnt_dev);
    KCHECK();
  }
  // 3. the cotangents of the next state: particles to slot order, fields
  //    to spectra
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const bool have_x1 = xbar1 != nullptr, have_P1 = Pbar1 != nullptr;
  if (np > 0 && (have_x1 || have_P1)) {
    double *tmp = ptmp;
    if (have_x1) {
      CK(cudaMemcpyAsync(tmp, xbar1, sizeof(double) * d * np, kin, ctx->st));
      k_rows_to_slot<<<grid_of(np), 256, 0, ctx->st>>>(tmp, xb1s, ctx->id, np, (int64_t)cap, d);
      KCHECK();
    }
    if (have_P1) {
      CK(cudaMemcpyAsync(tmp, Pbar1, sizeof(double) * 3 * np, kin, ctx->st));
      k_rows_to_slot<<<grid_of(np), 256, 0, ctx->st>>>(tmp, Pb1s, ctx->id, np, (int64_t)cap, 3);
      KCHECK();
    }
  }
  if (fbar1) CK(cudaMemcpyAsync(f1, fbar1, sizeof(double) * 9 * Ng, kin, ctx->st));
  else CK(cudaMemsetAsync(f1, 0, sizeof(double) * 9 * Ng, ctx->st));
  if ((e = field_real_to_complex(ctx, f1, Ys, 9))) return e;
  if ((e = fft_nd(ctx, Ys, 9, -1))) return e;
  CK(cudaMemsetAsync(Zs, 0, sizeof(double2) * 9 * Ng, ctx->st));
  // the generalised VJP at (j*, S^n): with_y adds the next state's
  // cotangents, Jbar_or_null the deposit's; writes jbar, and with
  // want_state the current state's cotangents (f0 and xb0s / Pb0s)
  auto apply = [&](const double *Jbar_in, bool with_y, bool want_state) -> int {
    int r;
    CK(cudaMemsetAsync(Fbar, 0, sizeof(double) * (d + 6) * Ng, ctx->st));
    if (np > 0) {
      const double *xb = with_y && have_x1 ? xb1s : nullptr;
      const double *Pb = with_y && have_P1 ? Pb1s : nullptr;
#define PIC_SADJ(DD)                                                                          \
  k_sadj_mu<DD><<<nb, kPT, 0, ctx->st>>>(pv, Jbar_in, pg, kc, kcd, vbs, jvs, jps, xb, Pb, mus, \
                                         ctx->cnt_dev);                                       \
  KCHECK();                                                                                   \
  k_sadj_records<DD><<<nb, kPT, 0, ctx->st>>>(pv, nd, pg, kc, vbs, mus, Pb, want_state ? 1 : 0, \
                                              Fbar, ctx->cnt_dev);                            \
  KCHECK();                                                                                   \
  if (want_state) {                                                                           \
    k_sadj_momentum<DD><<<nb, kPT, 0, ctx->st>>>(pv, nd, pg, kc, vbs, mus, Pb, Fbar, Pb0s,     \
                                                 ctx->cnt_dev);                               \
    KCHECK();                                                                                 \
    k_sadj_position<DD><<<nb, kPT, 0, ctx->st>>>(pv, nd, dnodes, ctx->A_real, Jbar_in, pg, kc, \
                                                 kcd, vbs, mus, xb, Pb, xb0s, ctx->cnt_dev);  \
    KCHECK();                                                                                 \
  }
      if (d == 1) {
        PIC_SADJ(1);
      } else if (d == 2) {
        PIC_SADJ(2);
      } else {
        PIC_SADJ(3);
      }
#undef PIC_SADJ
    }
    // records and next state back through the field step
    if ((r = field_real_to_complex(ctx, Fbar, Rs, d + 3))) return r;
    if ((r = fft_nd(ctx, Rs, d + 3, -1))) return r;
    if ((r = field_cn_state_adjoint(ctx, with_y ? Ys : Zs, Rs, Os, 1.0 / Ng))) return r;
    if ((r = fft_nd(ctx, Os, 12, +1))) return r;
    if ((r = field_complex_to_real(ctx, Os + (size_t)9 * Ng, jbar, 3, 1.0))) return r;
    if (want_state) {
      if ((r = field_complex_to_real(ctx, Os, f0, 9, 1.0))) return r;
      // A^n is also read in real space (records A^n and A^- at the particles)
      if ((r = lincomb(ctx, f0 + 2 * (size_t)Ng, f0 + 2 * (size_t)Ng, 1.0,
                       Fbar + (size_t)(d + 3) * Ng, 1.0, N3)))
        return r;
    }
    return PIC_OK;
  };
  auto status_of = [&](int *out) -> int {
    EvalCounters cnt;
    CK(cudaMemcpyAsync(&cnt, ctx->cnt_dev, sizeof cnt, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    *out = (int)cnt.status;
    return PIC_OK;
  };
  int stbits = 0;
  if ((e = status_of(&stbits))) return e;
  if (stbits) {
    ctx->err = "pic_step_vjp: inner particle solve failed at the converged current (status bits " +
               std::to_string(stbits) + ")";
    return PIC_EINNER;
  }
  // 4. rhs = G_j^T Sbar', then (I - H_j^T) lambda = rhs, H_j^T l the j-part of
  //    the VJP with the deposit's cotangent P l
  if ((e = apply(nullptr, true, false))) return e;
  CK(cudaMemcpyAsync(rhs, jbar, sizeof(double) * N3, cudaMemcpyDeviceToDevice, ctx->st));
  auto op = [&](const double *l, double *out) -> int {
    int r;
    if ((r = field_project_real(ctx, l, Jb, 3))) return r;
    if ((r = apply(Jb, false, false))) return r;
    return lincomb(ctx, out, l, 1.0, jbar, -1.0, N3);
  };
  int its = 0;
  e = gmres_solve(ctx, op, rhs, lam, gws, std::fmax(tol, 1e-12), &its);
  if (gmres_iters) *gmres_iters = its;
  if (e) return e;
  // 5. Sbar = G_S^T Sbar' + H_S^T lambda
  if ((e = field_project_real(ctx, lam, Jb, 3))) return e;
  if ((e = apply(Jb, true, true))) return e;
  if ((e = status_of(&stbits))) return e;
  if (stbits) {
    ctx->err = "pic_step_vjp: adjoint particle solve failed (status bits " +
               std::to_string(stbits) + ")";
    return PIC_EINNER;
  }
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (fbar0) CK(cudaMemcpyAsync(fbar0, f0, sizeof(double) * 9 * Ng, kout, ctx->st));
  if (np > 0 && (xbar0 || Pbar0)) {
    double *tmp = ptmp;
    if (xbar0) {
      k_rows_to_load<<<grid_of(np), 256, 0, ctx->st>>>(xb0s, tmp, ctx->id, np, (int64_t)cap, d);
      KCHECK();
      CK(cudaMemcpyAsync(xbar0, tmp, sizeof(double) * d * np, kout, ctx->st));
      CK(cudaStreamSynchronize(ctx->st));
    }
    if (Pbar0) {
      k_rows_to_load<<<grid_of(np), 256, 0, ctx->st>>>(Pb0s, tmp, ctx->id, np, (int64_t)cap, 3);
      KCHECK();
      CK(cudaMemcpyAsync(Pbar0, tmp, sizeof(double) * 3 * np, kout, ctx->st));
    }
  }
  CK(cudaStreamSynchronize(ctx->st));
  return PIC_OK;
}
