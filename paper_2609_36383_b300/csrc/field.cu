// field.cu -- spectral field step of one map evaluation and the mesh
// diagnostics.
//
//  * k_cn_update: Nyquist projection of the trial current (Eq.
//    nyquist-projector), continuity (Eq. cn-continuity), and the closed-form
//    solution of the CN potential system (Eq. CN-field) for every Fourier
//    mode: with a = dt/2, b = dt kappa^2 |k|^2 / 2 and source s,
//        psi' = ((1 - a b) psi - 2 b phi + s) / (1 + a b),  phi' = phi + a (psi' + psi),
//    and the same map for (A_c, U_c) with source dt kappa^2 sigma2 J_c.  It also
//    emits the spectra that the particle gather needs: i k phi^{1/2}, A^{n+1}
//    and (final pass) U^{n+1/2}.
//  * k_pack_nodes: after the inverse transforms, interleaves those fields
//    with A^n into one record per node in the particle real type, so a gather
//    reads one contiguous record per stencil node.
//  * Parseval reductions for the field energy (Eq. field-energy-section2), the
//    Gauss and Lorenz residuals (Eq. constraint-residuals) and the mesh side
//    of the work residual (Eq. work-diagnostic).
#include "pic_internal.cuh"
#include "csum.cuh"

#include <cmath>

namespace {

constexpr int kThreads = 256;

struct SpecGeom {
  int dim, Ng;
  int n[3], s[3];  // sizes and strides
  double twopi_L[3];
  int project;
};

SpecGeom spec_geom(const pic_ctx *ctx) {
  SpecGeom sg;
  sg.dim = ctx->g.dim;
  sg.Ng = ctx->g.Ng;
  int st = 1;
  for (int a = 0; a < 3; a++) {
    sg.n[a] = ctx->g.n[a];
    sg.s[a] = st;
    st *= ctx->g.n[a];
    sg.twopi_L[a] = 2.0 * M_PI / ctx->g.L[a];
  }
  sg.project = ctx->opt.project_nyquist;
  return sg;
}

// Derivative symbols of mode g (zero on an even-grid Nyquist index and in
// ignorable dimensions) and whether g lies on a Nyquist plane.
__device__ __forceinline__ bool mode_symbols(const SpecGeom &sg, int g, double k[3]) {
  bool nyq = false;
  for (int a = 0; a < 3; a++) {
    k[a] = 0.0;
    if (a >= sg.dim) continue;
    int N = sg.n[a];
    int idx = (g / sg.s[a]) % N;
    if (idx == N / 2) { nyq = true; continue; }  // N is a power of two, so even
    int kk = idx < N / 2 ? idx : idx - N;
    k[a] = sg.twopi_L[a] * kk;
  }
  return nyq;
}

__device__ __forceinline__ double2 cmul_i(double s, double2 z) {  // (i s) z
  return make_double2(-s * z.y, s * z.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 cscale(double s, double2 a) {
  return make_double2(s * a.x, s * a.y);
}

// One CN mode update for the pair (f, g) = (phi, psi) or (A_c, U_c).
__device__ __forceinline__ void cn_mode(double a, double b, double2 f, double2 gg, double2 src,
                                        double2 *f1, double2 *g1) {
  double inv = 1.0 / (1.0 + a * b);
  double c1 = (1.0 - a * b) * inv, c2 = -2.0 * b * inv;
  double2 gn = make_double2((c1 * gg.x + c2 * f.x + src.x * inv),
                            (c1 * gg.y + c2 * f.y + src.y * inv));
  *g1 = gn;
  *f1 = make_double2(f.x + a * (gn.x + gg.x), f.y + a * (gn.y + gg.y));
}

__global__ void k_r2c(const double *__restrict__ src, double2 *__restrict__ dst, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = make_double2(src[i], 0.0);
}

__global__ void k_c2r(const double2 *__restrict__ src, double *__restrict__ dst, size_t n,
                      double scale) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i].x * scale;
}

__global__ void k_project(double2 *f, SpecGeom sg, int ncomp) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= sg.Ng) return;
  double k[3];
  if (mode_symbols(sg, g, k) && sg.project)
    for (int c = 0; c < ncomp; c++) f[(size_t)c * sg.Ng + g] = make_double2(0.0, 0.0);
}

struct CnArgs {
  const double2 *jh, *rho, *phi, *psi, *A, *U;
  double2 *rho1, *phi1, *psi1, *A1, *U1;
  double2 *out;  // gather spectra: dim comps of i k phi^{1/2}, 3 of A^{n+1}, 3 of U^{1/2}
  double dt, kap2, sigma1, sigma2;
  int want_uhalf;
};

__global__ void k_cn_update(CnArgs p, SpecGeom sg) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= sg.Ng) return;
  const int Ng = sg.Ng, d = sg.dim;
  double k[3];
  bool nyq = mode_symbols(sg, g, k);
  const double2 z = make_double2(0.0, 0.0);
  if (nyq && sg.project) {
    p.rho1[g] = z; p.phi1[g] = z; p.psi1[g] = z;
    for (int c = 0; c < 3; c++) { p.A1[c * Ng + g] = z; p.U1[c * Ng + g] = z; }
    for (int c = 0; c < d + 3 + (p.want_uhalf ? 3 : 0); c++) p.out[(size_t)c * Ng + g] = z;
    return;
  }
  double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  double2 j[3] = {p.jh[g], p.jh[Ng + g], p.jh[2 * Ng + g]};
  // continuity: rho' = rho - dt (i k . j)
  double2 divj = cadd(cadd(cmul_i(k[0], j[0]), cmul_i(k[1], j[1])), cmul_i(k[2], j[2]));
  double2 rho0 = p.rho[g];
  double2 rho1 = make_double2(rho0.x - p.dt * divj.x, rho0.y - p.dt * divj.y);
  double2 rhoh = make_double2(0.5 * (rho0.x + rho1.x), 0.5 * (rho0.y + rho1.y));
  double a = 0.5 * p.dt, b = 0.5 * p.dt * p.kap2 * k2;
  double2 phi1, psi1;
  double2 phi0 = p.phi[g];
  cn_mode(a, b, phi0, p.psi[g], cscale(p.dt * p.kap2 * p.sigma1, rhoh), &phi1, &psi1);
  p.rho1[g] = rho1; p.phi1[g] = phi1; p.psi1[g] = psi1;
  double2 phih = make_double2(0.5 * (phi0.x + phi1.x), 0.5 * (phi0.y + phi1.y));
  for (int c = 0; c < d; c++) p.out[(size_t)c * Ng + g] = cmul_i(k[c], phih);
  for (int c = 0; c < 3; c++) {
    double2 A0 = p.A[c * Ng + g], U0 = p.U[c * Ng + g], A1, U1;
    cn_mode(a, b, A0, U0, cscale(p.dt * p.kap2 * p.sigma2, j[c]), &A1, &U1);
    p.A1[c * Ng + g] = A1;
    p.U1[c * Ng + g] = U1;
    p.out[(size_t)(d + c) * Ng + g] = A1;
    if (p.want_uhalf)
      p.out[(size_t)(d + 3 + c) * Ng + g] = make_double2(0.5 * (U0.x + U1.x), 0.5 * (U0.y + U1.y));
  }
}

// Node records [grad phi^{1/2} (d), A^n (3), A^{n+1} (3)] padded to nvp reals
// (a multiple of four), and U^{1/2} records padded to four reals.
template <typename T>
__global__ void k_pack_nodes(const double2 *__restrict__ spec, const double *__restrict__ A_n,
                             double *__restrict__ A1_real, T *__restrict__ nodes,
                             T *__restrict__ nodes_u, int Ng, int d, int nvp, double inv_ng,
                             int want_uhalf) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Ng) return;
  T *rec = nodes + (size_t)g * nvp;
  for (int c = 0; c < d; c++) rec[c] = (T)(spec[(size_t)c * Ng + g].x * inv_ng);
  for (int c = 0; c < 3; c++) {
    rec[d + c] = (T)A_n[(size_t)c * Ng + g];
    double a1 = spec[(size_t)(d + c) * Ng + g].x * inv_ng;
    rec[d + 3 + c] = (T)a1;
    A1_real[(size_t)c * Ng + g] = a1;
  }
  for (int c = d + 6; c < nvp; c++) rec[c] = (T)0;
  if (want_uhalf) {
    for (int c = 0; c < 3; c++)
      nodes_u[(size_t)g * 4 + c] = (T)(spec[(size_t)(d + 3 + c) * Ng + g].x * inv_ng);
    nodes_u[(size_t)g * 4 + 3] = (T)0;
  }
}

// phi^0 from Gauss (k^2 phi = sigma1 rho + i k . U) and psi^0 from the
// Lorenz gauge (psi = -kappa^2 i k . A); the k = 0 mode of phi is zero.
__global__ void k_initial_constraints(double2 *phi, double2 *psi, const double2 *rho,
                                      const double2 *A, const double2 *U, SpecGeom sg,
                                      double sigma1, double kap2) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= sg.Ng) return;
  const int Ng = sg.Ng;
  double k[3];
  bool nyq = mode_symbols(sg, g, k);
  double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  double2 divU = make_double2(0, 0), divA = make_double2(0, 0);
  for (int c = 0; c < 3; c++) {
    divU = cadd(divU, cmul_i(k[c], U[c * Ng + g]));
    divA = cadd(divA, cmul_i(k[c], A[c * Ng + g]));
  }
  bool zero = nyq && sg.project;
  if (k2 > 0.0 && !zero) {
    double2 r = rho[g];
    phi[g] = make_double2((sigma1 * r.x + divU.x) / k2, (sigma1 * r.y + divU.y) / k2);
  } else {
    phi[g] = make_double2(0, 0);
  }
  psi[g] = zero ? make_double2(0, 0) : cscale(-kap2, divA);
}

// ---- block reductions -------------------------------------------------------
template <int NQ>
__device__ void block_sum_write(double (&v)[NQ], double *out) {
  // compensated: each block writes NQ (sum, error) pairs
  __shared__ CSum sh[NQ][kThreads / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < NQ; q++) {
    CSum x = csum_warp(CSum{v[q], 0.0});
    if (lane == 0) sh[q][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    CSum t = csum_zero();
    for (int w = 0; w < (int)(blockDim.x / 32); w++) t = csum_merge(t, sh[threadIdx.x][w]);
    out[((size_t)blockIdx.x * NQ + threadIdx.x) * 2] = t.s;
    out[((size_t)blockIdx.x * NQ + threadIdx.x) * 2 + 1] = t.c;
  }
}

__global__ void k_energy_parts(const double2 *phi, const double2 *A, const double2 *U, SpecGeom sg,
                               double inv_2s1, double inv_2s2, double *out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (g < sg.Ng) {
    const int Ng = sg.Ng;
    double k[3];
    mode_symbols(sg, g, k);
    double2 ph = phi[g];
    double e2 = 0.0, b2 = 0.0;
    double2 Ah[3] = {A[g], A[Ng + g], A[2 * Ng + g]};
    for (int c = 0; c < 3; c++) {
      double2 E = cadd(cmul_i(-k[c], ph), cscale(-1.0, U[c * Ng + g]));
      e2 += E.x * E.x + E.y * E.y;
      int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
      double2 B = cadd(cmul_i(k[c1], Ah[c2]), cmul_i(-k[c2], Ah[c1]));
      b2 += B.x * B.x + B.y * B.y;
    }
    v[0] = e2 * inv_2s1 + b2 * inv_2s2;
  }
  block_sum_write<1>(v, out);
}

// Tangent of the field energy density: the derivative of |E|^2 / (2 sigma1)
// + |B|^2 / (2 sigma2) in the direction (dphi, dA, dU) is
// Re(conj(E) dE) / sigma1 + Re(conj(B) dB) / sigma2, with dE and dB the same
// linear maps of the tangent.
__global__ void k_energy_tangent_parts(const double2 *phi, const double2 *A, const double2 *U,
                                       const double2 *dphi, const double2 *dA,
                                       const double2 *dU, SpecGeom sg, double inv_2s1,
                                       double inv_2s2, double *out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (g < sg.Ng) {
    const int Ng = sg.Ng;
    double k[3];
    mode_symbols(sg, g, k);
    const double2 ph = phi[g], dph = dphi[g];
    double e2 = 0.0, b2 = 0.0;
    for (int c = 0; c < 3; c++) {
      const double2 E = cadd(cmul_i(-k[c], ph), cscale(-1.0, U[c * Ng + g]));
      const double2 dE = cadd(cmul_i(-k[c], dph), cscale(-1.0, dU[c * Ng + g]));
      e2 += E.x * dE.x + E.y * dE.y;
      const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
      const double2 B = cadd(cmul_i(k[c1], A[c2 * Ng + g]), cmul_i(-k[c2], A[c1 * Ng + g]));
      const double2 dB =
          cadd(cmul_i(k[c1], dA[c2 * Ng + g]), cmul_i(-k[c2], dA[c1 * Ng + g]));
      b2 += B.x * dB.x + B.y * dB.y;
    }
    v[0] = 2.0 * (e2 * inv_2s1 + b2 * inv_2s2);
  }
  block_sum_write<1>(v, out);
}

// Transpose of the field step's dependence on the trial current, mode by
// mode.  k_cn_update maps the transform j^ of the current to the gather
// spectra i k_c phi^{1/2} (c < dim) and A^{n+1}_c by a real symmetric matrix
// per mode: d(i k_c phi^{1/2}) = mu k_c (k . dj^) with
// mu = a dt^2 kappa^2 sigma1 / (4 (1 + a b)), and dA^{n+1}_c = g dj^_c with
// g = a dt kappa^2 sigma2 / (1 + a b) (a = dt/2, b = dt kappa^2 |k|^2 / 2;
// continuity enters through rho^{1/2}).  So the adjoint is the same matrix;
// `scale` folds in the 1/Ng of the inverse transform behind the records.
__global__ void k_cn_adjoint(const double2 *__restrict__ sbar, double2 *__restrict__ jbar,
                             SpecGeom sg, double dt, double kap2, double sigma1, double sigma2,
                             double scale) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= sg.Ng) return;
  const int Ng = sg.Ng, d = sg.dim;
  double k[3];
  const bool nyq = mode_symbols(sg, g, k);
  if (nyq && sg.project) {
    for (int c = 0; c < 3; c++) jbar[c * Ng + g] = make_double2(0.0, 0.0);
    return;
  }
  const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  const double a = 0.5 * dt, b = 0.5 * dt * kap2 * k2, inv = 1.0 / (1.0 + a * b);
  const double mu = a * inv * dt * dt * kap2 * sigma1 * 0.25, gam = a * inv * dt * kap2 * sigma2;
  double2 ks = make_double2(0.0, 0.0);  // sum_c k_c sbar_phi,c
  for (int c = 0; c < d; c++) ks = cadd(ks, cscale(k[c], sbar[(size_t)c * Ng + g]));
  for (int e = 0; e < 3; e++)
    jbar[e * Ng + g] =
        cscale(scale, cadd(cscale(mu * k[e], ks), cscale(gam, sbar[(size_t)(d + e) * Ng + g])));
}

// Transpose of the whole field step, mode by mode (the adjoint of a step).
// k_cn_update maps (phi, psi, A, U, rho, j^) of a mode to the next state
// (phi', psi', A', U', rho') and to the gather spectra (i k_c phi^{1/2},
// A'); its coefficients are real except for the factors i k, whose
// transpose under the real inner product of the real-space fields is -i k.
// ybar holds the cotangents of the next state [phi', psi', A' (3), U' (3),
// rho'] and rbar those of the gather spectra [i k phi^{1/2} (dim), A' (3)],
// both as forward transforms of real-space cotangents; out receives
// [phi, psi, A (3), U (3), rho, j^ (3)] times scale.  The 2 x 3 matrix of
// cn_mode is read off cn_mode itself (it is linear), so the transpose uses
// the forward step's own coefficients.
__global__ void k_cn_state_adjoint(const double2 *__restrict__ ybar,
                                   const double2 *__restrict__ rbar, double2 *__restrict__ out,
                                   SpecGeom sg, double dt, double kap2, double sigma1,
                                   double sigma2, double scale) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= sg.Ng) return;
  const int Ng = sg.Ng, d = sg.dim;
  const double2 z = make_double2(0.0, 0.0);
  double k[3];
  const bool nyq = mode_symbols(sg, g, k);
  if (nyq && sg.project) {  // the forward step zeroes every output of the mode
    for (int c = 0; c < 12; c++) out[(size_t)c * Ng + g] = z;
    return;
  }
  const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  const double a = 0.5 * dt, b = 0.5 * dt * kap2 * k2;
  // cn_mode: (f1, g1) = M (f, g, src) with M real; column q from input e_q
  double M[2][3];
  for (int q = 0; q < 3; q++) {
    const double2 f = make_double2(q == 0 ? 1.0 : 0.0, 0.0);
    const double2 gg = make_double2(q == 1 ? 1.0 : 0.0, 0.0);
    const double2 sr = make_double2(q == 2 ? 1.0 : 0.0, 0.0);
    double2 f1, g1;
    cn_mode(a, b, f, gg, sr, &f1, &g1);
    M[0][q] = f1.x;
    M[1][q] = g1.x;
  }
  auto mt = [&](int q, double2 f1b, double2 g1b) {  // row q of M^T (f1b, g1b)
    return cadd(cscale(M[0][q], f1b), cscale(M[1][q], g1b));
  };
  double2 jb[3] = {z, z, z};
  // vector potential: A' enters the next state and the gather records
  for (int c = 0; c < 3; c++) {
    const double2 Ab = cadd(ybar[(size_t)(2 + c) * Ng + g], rbar[(size_t)(d + c) * Ng + g]);
    const double2 Ub = ybar[(size_t)(5 + c) * Ng + g];
    out[(size_t)(2 + c) * Ng + g] = cscale(scale, mt(0, Ab, Ub));
    out[(size_t)(5 + c) * Ng + g] = cscale(scale, mt(1, Ab, Ub));
    jb[c] = cscale(dt * kap2 * sigma2, mt(2, Ab, Ub));
  }
  // scalar potential: phi^{1/2} = (phi + phi') / 2 feeds the records i k phi^{1/2}
  double2 phb = z;
  for (int c = 0; c < d; c++) phb = cadd(phb, cmul_i(-k[c], rbar[(size_t)c * Ng + g]));
  const double2 f1b = cadd(ybar[g], cscale(0.5, phb)), g1b = ybar[(size_t)Ng + g];
  out[g] = cscale(scale, cadd(cscale(0.5, phb), mt(0, f1b, g1b)));
  out[(size_t)Ng + g] = cscale(scale, mt(1, f1b, g1b));
  // source dt kap2 sigma1 rho^{1/2}; rho^{1/2} = rho - (dt/2) div j, rho' = rho - dt div j
  const double2 rhb = cscale(dt * kap2 * sigma1, mt(2, f1b, g1b));
  const double2 r1b = ybar[(size_t)8 * Ng + g];
  out[(size_t)8 * Ng + g] = cscale(scale, cadd(r1b, rhb));
  const double2 divb = cadd(cscale(-dt, r1b), cscale(-0.5 * dt, rhb));
  for (int c = 0; c < 3; c++) {
    jb[c] = cadd(jb[c], cmul_i(-k[c], divb));
    out[(size_t)(9 + c) * Ng + g] = cscale(scale, jb[c]);
  }
}

__global__ void k_constraint_parts(const double2 *phi, const double2 *psi, const double2 *rho,
                                   const double2 *A, const double2 *U, SpecGeom sg,
                                   double sigma1, double inv_kap2, double *out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (g < sg.Ng) {
    const int Ng = sg.Ng;
    double k[3];
    mode_symbols(sg, g, k);
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    double2 divU = make_double2(0, 0), divA = make_double2(0, 0);
    for (int c = 0; c < 3; c++) {
      divU = cadd(divU, cmul_i(k[c], U[c * Ng + g]));
      divA = cadd(divA, cmul_i(k[c], A[c * Ng + g]));
    }
    double2 ph = phi[g], r = rho[g], ps = psi[g];
    double2 RG = make_double2(k2 * ph.x - divU.x - sigma1 * r.x, k2 * ph.y - divU.y - sigma1 * r.y);
    double2 RL = make_double2(ps.x * inv_kap2 + divA.x, ps.y * inv_kap2 + divA.y);
    v[0] = RG.x * RG.x + RG.y * RG.y;
    v[1] = RL.x * RL.x + RL.y * RL.y;
  }
  block_sum_write<2>(v, out);
}

// sum_k Re(J_k conj(E_k)) with E^{1/2} = -i k phi^{1/2} - U^{1/2}
__global__ void k_mesh_work_parts(const double2 *Jh, const double2 *phi0, const double2 *phi1,
                                  const double2 *U0, const double2 *U1, SpecGeom sg,
                                  double *out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (g < sg.Ng) {
    const int Ng = sg.Ng;
    double k[3];
    mode_symbols(sg, g, k);
    double2 ph = make_double2(0.5 * (phi0[g].x + phi1[g].x), 0.5 * (phi0[g].y + phi1[g].y));
    double s = 0.0;
    for (int c = 0; c < 3; c++) {
      double2 Uh = make_double2(0.5 * (U0[c * Ng + g].x + U1[c * Ng + g].x),
                                0.5 * (U0[c * Ng + g].y + U1[c * Ng + g].y));
      double2 E = cadd(cmul_i(-k[c], ph), cscale(-1.0, Uh));
      double2 J = Jh[c * Ng + g];
      s += J.x * E.x + J.y * E.y;
    }
    v[0] = s;
  }
  block_sum_write<1>(v, out);
}

// (I - Q_a) f along one axis, where Q_a f = c (-1)^n on every line along a
// with c the alternating mean (1/N) sum_n f_n (-1)^n: the projection onto the
// modes with k_a = N_a/2.  The product of these factors over the active axes
// is the projector of Eq. nyquist-projector (the Q_a commute), so applying
// one kernel per axis projects a real mesh field without a Fourier round trip.
// One CTA per line; in-place when src == dst.
__global__ void k_nyq_axis(const double *src, double *dst, int Ng, int N, int stride) {
  __shared__ double sh[kThreads / 32];
  const int ln = blockIdx.x;
  const double *in = src + (size_t)blockIdx.y * Ng;
  double *out = dst + (size_t)blockIdx.y * Ng;
  const size_t base = (size_t)(ln % stride) + (size_t)(ln / stride) * stride * N;
  double s = 0.0;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    double v = in[base + (size_t)k * stride];
    s += (k & 1) ? -v : v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  double c = 0.0;
  for (int w = 0; w < (int)(blockDim.x / 32); w++) c += sh[w];
  c /= N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    size_t a = base + (size_t)k * stride;
    out[a] = in[a] - ((k & 1) ? -c : c);
  }
}

// sum_g H . E^{1/2} over the mesh in real space, with E^{1/2} = -grad phi^{1/2}
// - U^{1/2} read from the inverse-transformed gather spectra (real parts,
// scaled by 1/Ng)
__global__ void k_mesh_work_real(const double *H, const double2 *spec, int Ng, int d,
                                 double inv_ng, double *out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (g < Ng) {
    double s = 0.0;
    for (int c = 0; c < 3; c++) {
      double E = -spec[(size_t)(d + 3 + c) * Ng + g].x * inv_ng;
      if (c < d) E -= spec[(size_t)c * Ng + g].x * inv_ng;
      s += H[(size_t)c * Ng + g] * E;
    }
    v[0] = s;
  }
  block_sum_write<1>(v, out);
}

template <int NQ>
__global__ void k_sum_partials(const double *parts, int nblk, double *out) {
  // one block; fixed summation order for run-to-run reproducibility; the
  // block partials are (sum, error) pairs merged with compensation
  __shared__ CSum sh[NQ][kThreads];
  for (int q = 0; q < NQ; q++) {
    CSum t = csum_zero();
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
      t = csum_merge(t, CSum{parts[((size_t)b * NQ + q) * 2], parts[((size_t)b * NQ + q) * 2 + 1]});
    sh[q][threadIdx.x] = t;
  }
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int q = 0; q < NQ; q++) sh[q][threadIdx.x] = csum_merge(sh[q][threadIdx.x], sh[q][threadIdx.x + st]);
    __syncthreads();
  }
  if (threadIdx.x < NQ) out[threadIdx.x] = csum_value(sh[threadIdx.x][0]);
}

template <int NQ>
int finish_sum(pic_ctx *ctx, int nblk, double *host_out) {
  k_sum_partials<NQ><<<1, kThreads, 0, ctx->st>>>(ctx->red, nblk,
                                                   ctx->red + (size_t)nblk * NQ * 2);
  KCHECK();
  CK(cudaMemcpyAsync(ctx->red_host, ctx->red + (size_t)nblk * NQ * 2, sizeof(double) * NQ,
                     cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int q = 0; q < NQ; q++) host_out[q] = ctx->red_host[q];
  return PIC_OK;
}

// the queued form: the NQ sums land in dout[0 .. NQ) on the device
template <int NQ>
int queue_sum(pic_ctx *ctx, int nblk, double *dout) {
  k_sum_partials<NQ><<<1, kThreads, 0, ctx->st>>>(ctx->red, nblk, dout);
  KCHECK();
  return PIC_OK;
}

inline int blocks(size_t n) { return (int)((n + kThreads - 1) / kThreads); }

}  // namespace

int field_real_to_complex(pic_ctx *ctx, const double *src, double2 *dst, int ncomp) {
  size_t n = (size_t)ncomp * ctx->g.Ng;
  k_r2c<<<blocks(n), kThreads, 0, ctx->st>>>(src, dst, n);
  KCHECK();
  return PIC_OK;
}

int field_complex_to_real(pic_ctx *ctx, const double2 *src, double *dst, int ncomp,
                          double scale) {
  size_t n = (size_t)ncomp * ctx->g.Ng;
  k_c2r<<<blocks(n), kThreads, 0, ctx->st>>>(src, dst, n, scale);
  KCHECK();
  return PIC_OK;
}

int field_project_h(pic_ctx *ctx, double2 *f, int ncomp) {
  if (!ctx->opt.project_nyquist) return PIC_OK;
  k_project<<<blocks(ctx->g.Ng), kThreads, 0, ctx->st>>>(f, spec_geom(ctx), ncomp);
  KCHECK();
  return PIC_OK;
}

int field_cn_update_into(pic_ctx *ctx, const double2 *jh, const SpecState &in,
                         const SpecState &out, double2 *spec, int want_uhalf) {
  CnArgs p;
  p.jh = jh;
  p.rho = in.rho; p.phi = in.phi; p.psi = in.psi; p.A = in.A; p.U = in.U;
  p.rho1 = out.rho; p.phi1 = out.phi; p.psi1 = out.psi; p.A1 = out.A; p.U1 = out.U;
  p.out = spec;
  p.dt = ctx->dt;
  p.kap2 = ctx->opt.kappa * ctx->opt.kappa;
  p.sigma1 = ctx->opt.sigma1;
  p.sigma2 = ctx->opt.sigma2;
  p.want_uhalf = want_uhalf;
  k_cn_update<<<blocks(ctx->g.Ng), kThreads, 0, ctx->st>>>(p, spec_geom(ctx));
  KCHECK();
  return PIC_OK;
}

int field_cn_update(pic_ctx *ctx, const double2 *jh, int want_uhalf) {
  const SpecState in = {ctx->rho_h, ctx->phi_h, ctx->psi_h, ctx->A_h, ctx->U_h};
  const SpecState out = {ctx->rho1_h, ctx->phi1_h, ctx->psi1_h, ctx->A1_h, ctx->U1_h};
  return field_cn_update_into(ctx, jh, in, out, ctx->work_h, want_uhalf);
}

int field_pack_nodes(pic_ctx *ctx, int want_uhalf) {
  const int d = ctx->g.dim, Ng = ctx->g.Ng;
  int nc = d + 3 + (want_uhalf ? 3 : 0);
  int st = fft_nd(ctx, ctx->work_h, nc, +1);
  if (st) return st;
  double inv = 1.0 / Ng;
  if (ctx->eval_f32)  // FP32 records for the FP32 stage of an FP64 context
    k_pack_nodes<float><<<blocks(Ng), kThreads, 0, ctx->st>>>(
        ctx->work_h, ctx->A_real, ctx->A1_real, ctx->nodes_f, ctx->nodes_u_f, Ng, d,
        node_record_len(d), inv, want_uhalf);
  else if (ctx->rsize == 8)
    k_pack_nodes<double><<<blocks(Ng), kThreads, 0, ctx->st>>>(
        ctx->work_h, ctx->A_real, ctx->A1_real, (double *)ctx->nodes, (double *)ctx->nodes_u, Ng,
        d, node_record_len(d), inv, want_uhalf);
  else
    k_pack_nodes<float><<<blocks(Ng), kThreads, 0, ctx->st>>>(
        ctx->work_h, ctx->A_real, ctx->A1_real, (float *)ctx->nodes, (float *)ctx->nodes_u, Ng, d,
        node_record_len(d), inv, want_uhalf);
  KCHECK();
  return PIC_OK;
}

int field_pack_nodes_into(pic_ctx *ctx, double2 *spec, const double *A_n, double *A1_real,
                          double *nodes) {
  const int d = ctx->g.dim, Ng = ctx->g.Ng;
  int st = fft_nd(ctx, spec, d + 3, +1);
  if (st) return st;
  k_pack_nodes<double><<<blocks(Ng), kThreads, 0, ctx->st>>>(
      spec, A_n, A1_real, nodes, nullptr, Ng, d, node_record_len(d), 1.0 / Ng, 0);
  KCHECK();
  return PIC_OK;
}

int field_initial_constraints_into(pic_ctx *ctx, const SpecState &f) {
  k_initial_constraints<<<blocks(ctx->g.Ng), kThreads, 0, ctx->st>>>(
      f.phi, f.psi, f.rho, f.A, f.U, spec_geom(ctx), ctx->opt.sigma1,
      ctx->opt.kappa * ctx->opt.kappa);
  KCHECK();
  return PIC_OK;
}

int field_energy_tangent(pic_ctx *ctx, const SpecState &f, const SpecState &df, double *dW) {
  int nb = blocks(ctx->g.Ng);
  k_energy_tangent_parts<<<nb, kThreads, 0, ctx->st>>>(f.phi, f.A, f.U, df.phi, df.A, df.U,
                                                       spec_geom(ctx), 0.5 / ctx->opt.sigma1,
                                                       0.5 / ctx->opt.sigma2, ctx->red);
  KCHECK();
  double s;
  int e = finish_sum<1>(ctx, nb, &s);
  if (e) return e;
  *dW = s * ctx->g.dV / ctx->g.Ng;
  return PIC_OK;
}

int field_cn_adjoint(pic_ctx *ctx, const double2 *sbar, double2 *jbar, double scale) {
  k_cn_adjoint<<<blocks(ctx->g.Ng), kThreads, 0, ctx->st>>>(
      sbar, jbar, spec_geom(ctx), ctx->dt, ctx->opt.kappa * ctx->opt.kappa, ctx->opt.sigma1,
      ctx->opt.sigma2, scale);
  KCHECK();
  return PIC_OK;
}

int field_cn_state_adjoint(pic_ctx *ctx, const double2 *ybar, const double2 *rbar,
                           double2 *out, double scale) {
  k_cn_state_adjoint<<<blocks(ctx->g.Ng), kThreads, 0, ctx->st>>>(
      ybar, rbar, out, spec_geom(ctx), ctx->dt, ctx->opt.kappa * ctx->opt.kappa, ctx->opt.sigma1,
      ctx->opt.sigma2, scale);
  KCHECK();
  return PIC_OK;
}

int field_initial_constraints(pic_ctx *ctx) {
  k_initial_constraints<<<blocks(ctx->g.Ng), kThreads, 0, ctx->st>>>(
      ctx->phi_h, ctx->psi_h, ctx->rho_h, ctx->A_h, ctx->U_h, spec_geom(ctx), ctx->opt.sigma1,
      ctx->opt.kappa * ctx->opt.kappa);
  KCHECK();
  return PIC_OK;
}

int field_energy(pic_ctx *ctx, const double2 *phi_h, const double2 *A_h, const double2 *U_h,
                 double *W) {
  int nb = blocks(ctx->g.Ng);
  k_energy_parts<<<nb, kThreads, 0, ctx->st>>>(phi_h, A_h, U_h, spec_geom(ctx),
                                               0.5 / ctx->opt.sigma1, 0.5 / ctx->opt.sigma2,
                                               ctx->red);
  KCHECK();
  double s;
  int e = finish_sum<1>(ctx, nb, &s);
  if (e) return e;
  // Parseval for the unnormalised DFT: sum_g |f_g|^2 = sum_k |f_k|^2 / Ng
  *W = s * ctx->g.dV / ctx->g.Ng;
  return PIC_OK;
}

int field_energy_queued(pic_ctx *ctx, double *dout) {
  int nb = blocks(ctx->g.Ng);
  k_energy_parts<<<nb, kThreads, 0, ctx->st>>>(ctx->phi_h, ctx->A_h, ctx->U_h, spec_geom(ctx),
                                               0.5 / ctx->opt.sigma1, 0.5 / ctx->opt.sigma2,
                                               ctx->red);
  KCHECK();
  return queue_sum<1>(ctx, nb, dout);
}

int field_constraints_queued(pic_ctx *ctx, double *dout) {
  int nb = blocks(ctx->g.Ng);
  k_constraint_parts<<<nb, kThreads, 0, ctx->st>>>(ctx->phi_h, ctx->psi_h, ctx->rho_h, ctx->A_h,
                                                   ctx->U_h, spec_geom(ctx), ctx->opt.sigma1,
                                                   1.0 / (ctx->opt.kappa * ctx->opt.kappa),
                                                   ctx->red);
  KCHECK();
  return queue_sum<2>(ctx, nb, dout);
}

int field_constraints(pic_ctx *ctx, double *gauss_rms, double *lorenz_rms) {
  int nb = blocks(ctx->g.Ng);
  k_constraint_parts<<<nb, kThreads, 0, ctx->st>>>(ctx->phi_h, ctx->psi_h, ctx->rho_h, ctx->A_h,
                                                   ctx->U_h, spec_geom(ctx), ctx->opt.sigma1,
                                                   1.0 / (ctx->opt.kappa * ctx->opt.kappa),
                                                   ctx->red);
  KCHECK();
  double s[2];
  int e = finish_sum<2>(ctx, nb, s);
  if (e) return e;
  *gauss_rms = std::sqrt(s[0]) / ctx->g.Ng;
  *lorenz_rms = std::sqrt(s[1]) / ctx->g.Ng;
  return PIC_OK;
}

int field_project_real(pic_ctx *ctx, const double *src, double *dst, int ncomp) {
  const Geom &g = ctx->g;
  if (!ctx->opt.project_nyquist) {
    if (src != dst)
      CK(cudaMemcpyAsync(dst, src, sizeof(double) * ncomp * g.Ng, cudaMemcpyDeviceToDevice,
                         ctx->st));
    return PIC_OK;
  }
  int stride = 1;
  const double *in = src;
  for (int a = 0; a < g.dim; a++) {
    int N = g.n[a];
    int threads = N >= kThreads ? kThreads : (N < 32 ? 32 : N);
    dim3 grid(g.Ng / N, ncomp);
    k_nyq_axis<<<grid, threads, 0, ctx->st>>>(in, dst, g.Ng, N, stride);
    KCHECK();
    in = dst;
    stride *= N;
  }
  return PIC_OK;
}

// real-space mesh work of the last (final-pass) evaluation: H and the
// inverse-transformed gather spectra still in work_h
int field_mesh_work_real(pic_ctx *ctx, const double *H, double *work) {
  int nb = blocks(ctx->g.Ng);
  k_mesh_work_real<<<nb, kThreads, 0, ctx->st>>>(H, ctx->work_h, ctx->g.Ng, ctx->g.dim,
                                                 1.0 / ctx->g.Ng, ctx->red);
  KCHECK();
  double s;
  int e = finish_sum<1>(ctx, nb, &s);
  if (e) return e;
  *work = s * ctx->g.dV;
  return PIC_OK;
}

// mesh work sum_g J_orb . E^{1/2} dV of the last evaluation (Jorb_h holds the
// projected transform of J_orb; phi1_h, U1_h the candidate n+1 potentials)
int field_mesh_work_real_queued(pic_ctx *ctx, const double *H, double *dout) {
  int nb = blocks(ctx->g.Ng);
  k_mesh_work_real<<<nb, kThreads, 0, ctx->st>>>(H, ctx->work_h, ctx->g.Ng, ctx->g.dim,
                                                 1.0 / ctx->g.Ng, ctx->red);
  KCHECK();
  return queue_sum<1>(ctx, nb, dout);
}

int field_mesh_work(pic_ctx *ctx, double *work) {
  int nb = blocks(ctx->g.Ng);
  k_mesh_work_parts<<<nb, kThreads, 0, ctx->st>>>(ctx->Jorb_h, ctx->phi_h, ctx->phi1_h,
                                                  ctx->U_h, ctx->U1_h, spec_geom(ctx), ctx->red);
  KCHECK();
  double s;
  int e = finish_sum<1>(ctx, nb, &s);
  if (e) return e;
  *work = s * ctx->g.dV / ctx->g.Ng;
  return PIC_OK;
}
