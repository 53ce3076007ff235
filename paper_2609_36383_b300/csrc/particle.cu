// particle.cu -- particle side of the GM-HC-CN map evaluation.
//
// k_map<D, T> is the hot loop.  One thread owns one particle and runs its
// inner Picard iteration (Sec. 4.5) to convergence:
//   orbit x(s) = x^n + s dt vbar (Eq. rel-orbit), split at every crossed knot
//   of the quadratic B-spline (half-integer node coordinates), Gauss-Legendre
//   points on each piece (exact for the piecewise polynomials, Sec. 2.5) ->
//   gather of grad phi^{1/2} (Eq. orbit-gather-general), the orbit discrete
//   gradient D_i A (Eq. D-def), A^+ = A^{n+1}_h(x^{n+1}) ->
//   GM-HC canonical step (Eq. gmhc-step) with B_eff of K = D^T - D
//   (Eqs. D-split-skew, beff-KA) and the HC map (Def. hc-normalized) ->
//   orbit velocity from the two secant velocities (Eqs. Vdg, vbar-energy).
// After convergence the same thread deposits q vbar Sbar / dV with the final
// orbit velocity (Eq. orbit-current-energy), and on the final (verification)
// evaluation also accumulates the particle sides of the work and chain-rule
// diagnostics (Eqs. work-diagnostic, RA-diagnostic).
//
// Positions are an integer nearest-node index per active dimension plus an
// offset in node units in [-1/2, 1/2); the orbit is walked in that local
// frame, so the FP32 instantiation keeps its resolution anywhere in the box.
#include "pic_internal.cuh"

#include <cmath>

namespace {

constexpr int kPT = 128;     // particle kernel block size
constexpr int kMaxPieces = 16;

struct PGeom {
  int n[3], mask[3];
  int Ng, n0, n01;
  double dx[3], inv_dx[3], x0[3], L[3];
  double inv_dV;
};

PGeom pgeom(const pic_ctx *ctx) {
  PGeom p;
  for (int a = 0; a < 3; a++) {
    p.n[a] = ctx->g.n[a];
    p.mask[a] = ctx->g.n[a] - 1;
    p.dx[a] = ctx->g.dx[a];
    p.inv_dx[a] = 1.0 / ctx->g.dx[a];
    p.x0[a] = ctx->g.x0[a];
    p.L[a] = ctx->g.L[a];
  }
  p.Ng = ctx->g.Ng;
  p.n0 = ctx->g.n[0];
  p.n01 = ctx->g.n[0] * ctx->g.n[1];
  p.inv_dV = 1.0 / ctx->g.dV;
  return p;
}

inline int nblk(int64_t n) { return (int)((n + kPT - 1) / kPT); }

// quadratic B-spline weights of the three nodes b-1, b, b+1 for t = u - b in
// [-1/2, 1/2], and their derivatives with respect to u
template <typename T>
__device__ __forceinline__ void qspline(T t, T S[3], T dS[3]) {
  T a = T(0.5) - t, b = T(0.5) + t;
  S[0] = T(0.5) * a * a;
  S[1] = T(0.75) - t * t;
  S[2] = T(0.5) * b * b;
  dS[0] = -a;
  dS[1] = T(-2) * t;
  dS[2] = b;
}

template <typename T>
__device__ __forceinline__ void qspline_val(T t, T S[3]) {
  T a = T(0.5) - t, b = T(0.5) + t;
  S[0] = T(0.5) * a * a;
  S[1] = T(0.75) - t * t;
  S[2] = T(0.5) * b * b;
}

template <int D>
__device__ __forceinline__ int node_index(const PGeom &pg, const int cell[3], const int base[3],
                                          const int o[3]) {
  int g = (cell[0] + base[0] + o[0]) & pg.mask[0];
  if (D > 1) g += pg.n0 * ((cell[1] + base[1] + o[1]) & pg.mask[1]);
  if (D > 2) g += pg.n01 * ((cell[2] + base[2] + o[2]) & pg.mask[2]);
  return g;
}

// Walks the knot-split pieces of the straight orbit u(s) = off + s del,
// s in [0, 1], calling f(base, sa, sb) on each piece, where base is the node
// (relative to the particle's cell) nearest to u inside the piece.  Returns
// false if the orbit has more pieces than kMaxPieces.
template <int D, typename T, typename F>
__device__ __forceinline__ bool walk_orbit(const T off[3], const T del[3], F &f) {
  T d0[3], stp[3], nxt[3];
  int kc[3];
#pragma unroll
  for (int l = 0; l < D; l++) {
    kc[l] = 0;
    if (del[l] == T(0)) {
      nxt[l] = T(2);
      stp[l] = T(0);
      d0[l] = T(0);
      continue;
    }
    d0[l] = del[l] > T(0) ? T(0.5) - off[l] : off[l] + T(0.5);
    if (d0[l] <= T(0)) d0[l] = T(1);
    stp[l] = T(1) / fabs(del[l]);
    nxt[l] = d0[l] * stp[l];
  }
  T sa = T(0);
#pragma unroll 1
  for (int p = 0; p < kMaxPieces; p++) {
    T sb = T(1);
#pragma unroll
    for (int l = 0; l < D; l++) sb = fmin(sb, nxt[l]);
    if (sb > sa) {
      int base[3] = {0, 0, 0};
      T sm = T(0.5) * (sa + sb);
#pragma unroll
      for (int l = 0; l < D; l++) base[l] = (int)floor(off[l] + sm * del[l] + T(0.5));
      f(base, sa, sb);
    }
    if (sb >= T(1)) return true;
#pragma unroll
    for (int l = 0; l < D; l++)
      if (nxt[l] <= sb) {
        kc[l]++;
        nxt[l] = (d0[l] + T(kc[l])) * stp[l];
      }
    sa = sb;
  }
  return false;
}

// Orbit gather of grad phi^{1/2} and the discrete gradient D (3 x D) from
// the node records [gphi(D), A^n(3), A^{n+1}(3)].
template <int D, typename T>
struct GatherOrbit {
  const T *__restrict__ nodes;
  const PGeom *pg;
  const StepConst *sc;
  int cell[3];
  T off[3], del[3];
  T gphi[3];
  T Dm[3][3];
  int pieces;
  __device__ __forceinline__ void operator()(const int base[3], T sa, T sb) {
    constexpr int NV = D + 6;
    const T len = sb - sa;
    pieces++;
#pragma unroll 1
    for (int qp = 0; qp < sc->ngl; qp++) {
      const T s = sa + len * (T)sc->gl_t[qp];
      const T wt = len * (T)sc->gl_w[qp];
      T S[3][3], dS[3][3];
#pragma unroll
      for (int l = 0; l < D; l++) {
        qspline<T>(off[l] + s * del[l] - T(base[l]), S[l], dS[l]);
#pragma unroll
        for (int k = 0; k < 3; k++) dS[l][k] *= (T)pg->inv_dx[l];
      }
      const T s0 = T(1) - s;
#pragma unroll
      for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
#pragma unroll
        for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
#pragma unroll
          for (int ox = 0; ox < 3; ox++) {
            const int o[3] = {ox - 1, oy - 1, oz - 1};
            const int g = node_index<D>(*pg, cell, base, o);
            const T *rec = nodes + (size_t)g * NV;
            T Sx = S[0][ox], Sy = D > 1 ? S[1][oy] : T(1), Sz = D > 2 ? S[2][oz] : T(1);
            T w = wt * Sx * Sy * Sz;
            T dSw[3];
            dSw[0] = wt * dS[0][ox] * Sy * Sz;
            if (D > 1) dSw[1] = wt * Sx * dS[1][oy] * Sz;
            if (D > 2) dSw[2] = wt * Sx * Sy * dS[2][oz];
#pragma unroll
            for (int c = 0; c < D; c++) gphi[c] += w * __ldg(rec + c);
#pragma unroll
            for (int c = 0; c < 3; c++) {
              T Ac = s0 * __ldg(rec + D + c) + s * __ldg(rec + D + 3 + c);
#pragma unroll
              for (int j = 0; j < D; j++) Dm[c][j] += Ac * dSw[j];
            }
          }
    }
  }
};

// Deposit of q vbar Sbar / dV, optionally with the final-pass gathers
// (grad phi^{1/2}, U^{1/2}, D) used by the work and chain-rule diagnostics.
template <int D, typename T, bool FINAL>
struct DepositOrbit {
  const T *__restrict__ nodes;
  const T *__restrict__ nodes_u;
  double *__restrict__ J;
  const PGeom *pg;
  const StepConst *sc;
  int cell[3];
  T off[3], del[3];
  T qv[3];  // q vbar / dV
  T gphi[3], Ubar[3], Dm[3][3];
  int pieces;
  __device__ __forceinline__ void operator()(const int base[3], T sa, T sb) {
    constexpr int NN = D == 1 ? 3 : (D == 2 ? 9 : 27);
    constexpr int NV = D + 6;
    pieces++;
    T Sb[NN];
#pragma unroll
    for (int k = 0; k < NN; k++) Sb[k] = T(0);
    const T len = sb - sa;
#pragma unroll 1
    for (int qp = 0; qp < sc->ngl; qp++) {
      const T s = sa + len * (T)sc->gl_t[qp];
      const T wt = len * (T)sc->gl_w[qp];
      T S[3][3], dS[3][3];
#pragma unroll
      for (int l = 0; l < D; l++) {
        qspline<T>(off[l] + s * del[l] - T(base[l]), S[l], dS[l]);
#pragma unroll
        for (int k = 0; k < 3; k++) dS[l][k] *= (T)pg->inv_dx[l];
      }
      const T s0 = T(1) - s;
#pragma unroll
      for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
#pragma unroll
        for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
#pragma unroll
          for (int ox = 0; ox < 3; ox++) {
            T Sx = S[0][ox], Sy = D > 1 ? S[1][oy] : T(1), Sz = D > 2 ? S[2][oz] : T(1);
            T w = wt * Sx * Sy * Sz;
            Sb[ox + 3 * (oy + 3 * oz)] += w;
            if (FINAL) {
              const int o[3] = {ox - 1, oy - 1, oz - 1};
              const int g = node_index<D>(*pg, cell, base, o);
              const T *rec = nodes + (size_t)g * NV;
              const T *ru = nodes_u + (size_t)g * 3;
              T dSw[3];
              dSw[0] = wt * dS[0][ox] * Sy * Sz;
              if (D > 1) dSw[1] = wt * Sx * dS[1][oy] * Sz;
              if (D > 2) dSw[2] = wt * Sx * Sy * dS[2][oz];
#pragma unroll
              for (int c = 0; c < D; c++) gphi[c] += w * __ldg(rec + c);
#pragma unroll
              for (int c = 0; c < 3; c++) {
                Ubar[c] += w * __ldg(ru + c);
                T Ac = s0 * __ldg(rec + D + c) + s * __ldg(rec + D + 3 + c);
#pragma unroll
                for (int j = 0; j < D; j++) Dm[c][j] += Ac * dSw[j];
              }
            }
          }
    }
#pragma unroll
    for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
#pragma unroll
      for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
#pragma unroll
        for (int ox = 0; ox < 3; ox++) {
          const int o[3] = {ox - 1, oy - 1, oz - 1};
          const int g = node_index<D>(*pg, cell, base, o);
          const T sbv = Sb[ox + 3 * (oy + 3 * oz)];
#pragma unroll
          for (int c = 0; c < 3; c++) atomicAdd(J + (size_t)c * pg->Ng + g, (double)(qv[c] * sbv));
        }
  }
};

// A_h(u) at u = off + del (node coordinates relative to the cell), reading
// three components at stride `stride` from records of `rec_len` values
template <int D, typename T, typename S>
__device__ __forceinline__ void point_interp(const PGeom &pg, const int cell[3], const T u[3],
                                             const S *__restrict__ F, int rec_len, int first,
                                             size_t comp_stride, T out[3]) {
  int base[3] = {0, 0, 0};
  T Sw[3][3];
#pragma unroll
  for (int l = 0; l < D; l++) {
    base[l] = (int)floor(u[l] + T(0.5));
    qspline_val<T>(u[l] - T(base[l]), Sw[l]);
  }
  out[0] = out[1] = out[2] = T(0);
#pragma unroll
  for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
#pragma unroll
    for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
#pragma unroll
      for (int ox = 0; ox < 3; ox++) {
        const int o[3] = {ox - 1, oy - 1, oz - 1};
        const int g = node_index<D>(pg, cell, base, o);
        T w = Sw[0][ox] * (D > 1 ? Sw[1][oy] : T(1)) * (D > 2 ? Sw[2][oz] : T(1));
#pragma unroll
        for (int c = 0; c < 3; c++)
          out[c] += w * (T)__ldg(F + (size_t)g * rec_len + first + c * comp_stride);
      }
}

// GM-HC canonical step (Eq. gmhc-step) and orbit velocity (Eq. vbar-energy).
// gamma_n = gamma(p^n); Dm columns beyond D are zero and not read.
template <int D, typename T>
__device__ __forceinline__ void gmhc_push(const T Pn[3], const T Am[3], const T Ap[3],
                                          const T gphi[3], const T Dm[3][3], const T vb[3],
                                          T q, T m, T kap, T dt, T gamma_n, T vn[3], T Pn1[3]) {
  T Aep[3], com[3], pm[3];
  const T hq = T(0.5) * q * dt;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    Aep[c] = T(0.5) * (Am[c] + Ap[c]);
    T Dv = T(0);
#pragma unroll
    for (int j = 0; j < D; j++) Dv += Dm[c][j] * vb[j];
    com[c] = hq * (Dv - (c < D ? gphi[c] : T(0)));
    pm[c] = Pn[c] - q * Aep[c] + com[c];
  }
  // B_eff = (K_23, -K_13, K_12) with K = D^T - D, i.e. K_lj = D_jl - D_lj
  auto Dat = [&](int r, int c) -> T { return c < D ? Dm[r][c] : T(0); };
  T B[3];
  B[0] = Dat(2, 1) - Dat(1, 2);
  B[1] = -(Dat(2, 0) - Dat(0, 2));
  B[2] = Dat(1, 0) - Dat(0, 1);
  // HC magnetic map in u = p / (m kappa), Def. hc-normalized
  const T mk = m * kap, inv_mk = T(1) / mk;
  const T a = q * dt / (T(2) * m);
  T um[3], tau[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    um[c] = pm[c] * inv_mk;
    tau[c] = a * B[c];
  }
  const T u2 = um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
  const T gm2 = T(1) + u2;
  const T tau2 = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
  const T sig = gm2 - tau2;
  const T ut = um[0] * tau[0] + um[1] * tau[1] + um[2] * tau[2];
  const T gHC = sqrt(T(0.5) * (sig + sqrt(sig * sig + T(4) * (tau2 + ut * ut))));
  const T igHC = T(1) / gHC;
  T t[3];
#pragma unroll
  for (int c = 0; c < 3; c++) t[c] = tau[c] * igHC;
  const T t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  const T f = T(2) / (T(1) + t2);
  T us[3], up[3];
  us[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
  us[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
  us[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
  up[0] = um[0] + f * (us[1] * t[2] - us[2] * t[1]);
  up[1] = um[1] + f * (us[2] * t[0] - us[0] * t[2]);
  up[2] = um[2] + f * (us[0] * t[1] - us[1] * t[0]);
  T pp[3], pn[3], pn1[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    pp[c] = mk * up[c];
    Pn1[c] = pp[c] + q * Aep[c] + com[c];
    pn[c] = Pn[c] - q * Am[c];
    pn1[c] = Pn1[c] - q * Ap[c];
  }
  // secant velocities (Eq. Vdg); |p+| = |p-| (Eq. magnetic-kinetic-zero), so
  // gamma(p+) = gamma(p-) = sqrt(1 + |u-|^2)
  const T g_m = sqrt(gm2);
  const T ik2 = inv_mk * inv_mk;
  const T g_n1 = sqrt(T(1) + (pn1[0] * pn1[0] + pn1[1] * pn1[1] + pn1[2] * pn1[2]) * ik2);
  const T cm = T(0.5) / (m * (g_m + gamma_n));
  const T cp = T(0.5) / (m * (g_n1 + g_m));
#pragma unroll
  for (int c = 0; c < 3; c++) vn[c] = cm * (pm[c] + pn[c]) + cp * (pn1[c] + pp[c]);
}

template <typename T>
struct PView {
  int64_t np, cap;
  const int32_t *cell;
  const T *off, *P, *Am, *v0;
  const double *w;
  const int32_t *sp;
  T *vbar, *Pnew;
  int32_t *iters;
};

template <int NQ>
__device__ __forceinline__ void block_sums(double (&v)[NQ], double *out) {
  __shared__ double sh[NQ][kPT / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; q++) {
    double x = v[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[q][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double s = 0.0;
    for (int w = 0; w < kPT / 32; w++) s += sh[threadIdx.x][w];
    out[(size_t)blockIdx.x * NQ + threadIdx.x] = s;
  }
}

template <int D, typename T>
__global__ void __launch_bounds__(kPT)
k_map(PView<T> pv, const T *__restrict__ nodes, const T *__restrict__ nodes_u,
      double *__restrict__ J, PGeom pg, StepConst sc, int final_pass,
      EvalCounters *__restrict__ cnt, double *__restrict__ psum) {
  const int64_t i = blockIdx.x * (int64_t)kPT + threadIdx.x;
  const bool active = i < pv.np;
  double work = 0.0, chain = 0.0;
  int iters = 0, npieces = 0;
  unsigned int st = 0;
  if (active) {
    const int64_t cap = pv.cap;
    const int s_id = pv.sp[i];
    const T q = (T)(pv.w[i] * sc.qs[s_id]), m = (T)(pv.w[i] * sc.ms[s_id]);
    const T kap = (T)sc.kappa, dt = (T)sc.dt;
    int cell[3] = {0, 0, 0};
    T off[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int l = 0; l < D; l++) {
      cell[l] = pv.cell[l * cap + i];
      off[l] = pv.off[l * cap + i];
    }
    T Pn[3], Am[3], vb[3], Pn1[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      Pn[c] = pv.P[c * cap + i];
      Am[c] = pv.Am[c * cap + i];
      vb[c] = pv.v0[c * cap + i];
      Pn1[c] = Pn[c];
    }
    T pnv[3];
#pragma unroll
    for (int c = 0; c < 3; c++) pnv[c] = Pn[c] - q * Am[c];
    const T gamma_n =
        sqrt(T(1) + (pnv[0] * pnv[0] + pnv[1] * pnv[1] + pnv[2] * pnv[2]) / (m * m * kap * kap));
    const T tau_r = (T)sc.tau_r, tau_a = (T)sc.tau_a;
    bool conv = false;
    int it;
#pragma unroll 1
    for (it = 1; it <= sc.inner_max; it++) {
      GatherOrbit<D, T> go;
      go.nodes = nodes;
      go.pg = &pg;
      go.sc = &sc;
      go.pieces = 0;
#pragma unroll
      for (int l = 0; l < 3; l++) {
        go.cell[l] = cell[l];
        go.off[l] = off[l];
        go.del[l] = l < D ? dt * vb[l] * (T)pg.inv_dx[l] : T(0);
        go.gphi[l] = T(0);
        go.Dm[l][0] = go.Dm[l][1] = go.Dm[l][2] = T(0);
      }
      bool ok = walk_orbit<D, T>(go.off, go.del, go);
      npieces += go.pieces;
      if (!ok) {
        st |= PIC_ST_PIECES;
        break;
      }
      T u1[3], Ap[3];
#pragma unroll
      for (int l = 0; l < 3; l++) u1[l] = go.off[l] + go.del[l];
      point_interp<D, T, T>(pg, cell, u1, nodes, D + 6, D + 3, 1, Ap);
      T vn[3], Pc[3];
      gmhc_push<D, T>(Pn, Am, Ap, go.gphi, go.Dm, vb, q, m, kap, dt, gamma_n, vn, Pc);
      T diff = T(0), nrm = T(0), v2 = T(0);
      bool fin = true;
#pragma unroll
      for (int c = 0; c < 3; c++) {
        fin = fin && isfinite(vn[c]);
        diff = fmax(diff, fabs(vn[c] - vb[c]));
        nrm = fmax(nrm, fabs(vn[c]));
        v2 += vn[c] * vn[c];
      }
      if (!fin) { st |= PIC_ST_NONFINITE; break; }
      if (sqrt(v2) >= kap) { st |= PIC_ST_SUPERLUM; break; }
#pragma unroll
      for (int c = 0; c < 3; c++) {
        vb[c] = vn[c];
        Pn1[c] = Pc[c];
      }
      if (diff <= tau_a + tau_r * nrm) { conv = true; break; }
    }
    if (!conv && st == 0) st |= PIC_ST_NOCONV;
    iters = conv ? it : -1;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      pv.vbar[c * cap + i] = vb[c];
      pv.Pnew[c * cap + i] = Pn1[c];
    }
    pv.iters[i] = iters;
    if (conv) {
      const T qdv = q * (T)pg.inv_dV;
      if (!final_pass) {
        DepositOrbit<D, T, false> dp;
        dp.nodes = nodes; dp.nodes_u = nodes_u; dp.J = J; dp.pg = &pg; dp.sc = &sc;
        dp.pieces = 0;
#pragma unroll
        for (int l = 0; l < 3; l++) {
          dp.cell[l] = cell[l];
          dp.off[l] = off[l];
          dp.del[l] = l < D ? dt * vb[l] * (T)pg.inv_dx[l] : T(0);
          dp.qv[l] = qdv * vb[l];
        }
        if (!walk_orbit<D, T>(dp.off, dp.del, dp)) st |= PIC_ST_PIECES;
        npieces += dp.pieces;
      } else {
        DepositOrbit<D, T, true> dp;
        dp.nodes = nodes; dp.nodes_u = nodes_u; dp.J = J; dp.pg = &pg; dp.sc = &sc;
        dp.pieces = 0;
#pragma unroll
        for (int l = 0; l < 3; l++) {
          dp.cell[l] = cell[l];
          dp.off[l] = off[l];
          dp.del[l] = l < D ? dt * vb[l] * (T)pg.inv_dx[l] : T(0);
          dp.qv[l] = qdv * vb[l];
          dp.gphi[l] = dp.Ubar[l] = T(0);
          dp.Dm[l][0] = dp.Dm[l][1] = dp.Dm[l][2] = T(0);
        }
        if (!walk_orbit<D, T>(dp.off, dp.del, dp)) st |= PIC_ST_PIECES;
        npieces += dp.pieces;
        T u1[3], Ap[3];
#pragma unroll
        for (int l = 0; l < 3; l++) u1[l] = dp.off[l] + dp.del[l];
        point_interp<D, T, T>(pg, cell, u1, nodes, D + 6, D + 3, 1, Ap);
#pragma unroll
        for (int c = 0; c < 3; c++) {
          T Dv = T(0);
#pragma unroll
          for (int j = 0; j < D; j++) Dv += dp.Dm[c][j] * vb[j];
          T Eb = -(c < D ? dp.gphi[c] : T(0)) - dp.Ubar[c];
          work += (double)(q * vb[c] * Eb);
          T RA = Ap[c] - Am[c] - dt * (dp.Ubar[c] + Dv);
          chain += (double)RA * (double)RA;
        }
      }
    }
  }
  // counters
  if (st) atomicOr(&cnt->status, st);
  {
    double v[4] = {work, chain, (double)(iters > 0 ? iters : 0), (double)npieces};
    block_sums<4>(v, psum);
  }
  int mx = iters;
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(&cnt->inner_max, mx);
}

// ---- simple per-particle kernels -------------------------------------------
template <int D, typename T>
__global__ void k_load(int64_t n, int64_t cap, const double *__restrict__ x,
                       const double *__restrict__ uP, int canonical, const double *__restrict__ w,
                       const int32_t *__restrict__ sp, PGeom pg, int32_t *cell, T *off, T *P,
                       double *u_in, double *wo, int32_t *spo, int64_t *id) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int l = 0; l < D; l++) {
    double u = (x[l * n + i] - pg.x0[l]) * pg.inv_dx[l];
    double nn = (double)pg.n[l];
    u -= nn * floor(u / nn);
    int c = (int)floor(u + 0.5);
    double o = u - (double)c;
    if (c >= pg.n[l]) c -= pg.n[l];
    cell[l * cap + i] = c;
    off[l * cap + i] = (T)o;
  }
  for (int c = 0; c < 3; c++) {
    if (canonical) P[c * cap + i] = (T)uP[c * n + i];
    else u_in[c * cap + i] = uP[c * n + i];
  }
  wo[i] = w[i];
  spo[i] = sp ? sp[i] : 0;
  id[i] = i;
}

template <int D, typename T>
__global__ void k_form_P(PView<T> pv, T *P, const double *__restrict__ u_in,
                         const double *__restrict__ A, PGeom pg, StepConst sc) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np) return;
  int cell[3] = {0, 0, 0};
  double off[3] = {0, 0, 0};
  for (int l = 0; l < D; l++) {
    cell[l] = pv.cell[l * pv.cap + i];
    off[l] = (double)pv.off[l * pv.cap + i];
  }
  double Ax[3];
  point_interp<D, double, double>(pg, cell, off, A, 1, 0, (size_t)pg.Ng, Ax);
  int s = pv.sp[i];
  double q = pv.w[i] * sc.qs[s], m = pv.w[i] * sc.ms[s];
  for (int c = 0; c < 3; c++) P[c * pv.cap + i] = (T)(m * u_in[c * pv.cap + i] + q * Ax[c]);
}

template <int D, typename T>
__global__ void k_point_deposit(PView<T> pv, const double *__restrict__ A, PGeom pg,
                                StepConst sc, double *rho, double *J) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np) return;
  int cell[3] = {0, 0, 0};
  double off[3] = {0, 0, 0};
  for (int l = 0; l < D; l++) {
    cell[l] = pv.cell[l * pv.cap + i];
    off[l] = (double)pv.off[l * pv.cap + i];
  }
  double Ax[3];
  point_interp<D, double, double>(pg, cell, off, A, 1, 0, (size_t)pg.Ng, Ax);
  int s = pv.sp[i];
  double q = pv.w[i] * sc.qs[s], m = pv.w[i] * sc.ms[s];
  double p[3], p2 = 0.0;
  for (int c = 0; c < 3; c++) {
    p[c] = (double)pv.P[c * pv.cap + i] - q * Ax[c];
    p2 += p[c] * p[c];
  }
  double gam = sqrt(1.0 + p2 / (m * m * sc.kappa * sc.kappa));
  double Sw[3][3];
  for (int l = 0; l < D; l++) qspline_val<double>(off[l], Sw[l]);
  for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
    for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
      for (int ox = 0; ox < 3; ox++) {
        const int base[3] = {0, 0, 0};
        const int o[3] = {ox - 1, oy - 1, oz - 1};
        int g = node_index<D>(pg, cell, base, o);
        double S = Sw[0][ox] * (D > 1 ? Sw[1][oy] : 1.0) * (D > 2 ? Sw[2][oz] : 1.0);
        double qs = q * S * pg.inv_dV;
        atomicAdd(rho + g, qs);
        for (int c = 0; c < 3; c++) atomicAdd(J + (size_t)c * pg.Ng + g, qs * p[c] / (m * gam));
      }
}

template <int D, typename T>
__global__ void k_step_start(PView<T> pv, T *Am, T *v0, const double *__restrict__ A, PGeom pg,
                             StepConst sc) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np) return;
  int cell[3] = {0, 0, 0};
  double off[3] = {0, 0, 0};
  for (int l = 0; l < D; l++) {
    cell[l] = pv.cell[l * pv.cap + i];
    off[l] = (double)pv.off[l * pv.cap + i];
  }
  double Ax[3];
  point_interp<D, double, double>(pg, cell, off, A, 1, 0, (size_t)pg.Ng, Ax);
  int s = pv.sp[i];
  double q = pv.w[i] * sc.qs[s], m = pv.w[i] * sc.ms[s];
  double p[3], p2 = 0.0;
  for (int c = 0; c < 3; c++) {
    T a = (T)Ax[c];
    Am[c * pv.cap + i] = a;
    p[c] = (double)pv.P[c * pv.cap + i] - q * (double)a;
    p2 += p[c] * p[c];
  }
  double gam = sqrt(1.0 + p2 / (m * m * sc.kappa * sc.kappa));
  for (int c = 0; c < 3; c++) v0[c * pv.cap + i] = (T)(p[c] / (m * gam));
}

template <int D, typename T>
__global__ void k_commit(int64_t np, int64_t cap, int32_t *cell, T *off, T *P,
                         const T *__restrict__ vbar, const T *__restrict__ Pnew, PGeom pg,
                         double dt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  for (int l = 0; l < D; l++) {
    T u = off[l * cap + i] + (T)dt * vbar[l * cap + i] * (T)pg.inv_dx[l];
    T sh = floor(u + T(0.5));
    int c = cell[l * cap + i] + (int)sh;
    cell[l * cap + i] = c & pg.mask[l];
    off[l * cap + i] = u - sh;
  }
  for (int c = 0; c < 3; c++) P[c * cap + i] = Pnew[c * cap + i];
}

// kinetic energy m kappa^2 (gamma - 1) = |p|^2 / (m (gamma + 1)), p = P - q A_h(x)
template <int D, typename T>
__global__ void __launch_bounds__(kPT)
k_kinetic(PView<T> pv, const double *__restrict__ A, PGeom pg, StepConst sc, double *psum) {
  int64_t i = blockIdx.x * (int64_t)kPT + threadIdx.x;
  double v[1] = {0.0};
  if (i < pv.np) {
    int cell[3] = {0, 0, 0};
    double off[3] = {0, 0, 0};
    for (int l = 0; l < D; l++) {
      cell[l] = pv.cell[l * pv.cap + i];
      off[l] = (double)pv.off[l * pv.cap + i];
    }
    double Ax[3];
    point_interp<D, double, double>(pg, cell, off, A, 1, 0, (size_t)pg.Ng, Ax);
    int s = pv.sp[i];
    double q = pv.w[i] * sc.qs[s], m = pv.w[i] * sc.ms[s];
    double p2 = 0.0;
    for (int c = 0; c < 3; c++) {
      double p = (double)pv.P[c * pv.cap + i] - q * Ax[c];
      p2 += p * p;
    }
    double gam = sqrt(1.0 + p2 / (m * m * sc.kappa * sc.kappa));
    v[0] = p2 / (m * (gam + 1.0));
  }
  block_sums<1>(v, psum);
}

template <int D, typename T>
__global__ void k_export(PView<T> pv, const int64_t *__restrict__ id, PGeom pg, double *x,
                         double *P, double *w, int32_t *sp) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np) return;
  int64_t j = id[i], n = pv.np;
  if (x)
    for (int l = 0; l < D; l++) {
      double u = (double)pv.cell[l * pv.cap + i] + (double)pv.off[l * pv.cap + i];
      if (u < 0.0) u += (double)pg.n[l];
      x[l * n + j] = pg.x0[l] + u * pg.dx[l];
    }
  if (P)
    for (int c = 0; c < 3; c++) P[c * n + j] = (double)pv.P[c * pv.cap + i];
  if (w) w[j] = pv.w[i];
  if (sp) sp[j] = pv.sp[i];
}

template <typename T>
__global__ void k_export_eval(int64_t np, int64_t cap, const int64_t *__restrict__ id,
                              const T *vbar, const T *Pnew, const int32_t *iters, double *vo,
                              double *Po, int32_t *io) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  int64_t j = id[i];
  for (int c = 0; c < 3; c++) {
    if (vo) vo[c * np + j] = (double)vbar[c * cap + i];
    if (Po) Po[c * np + j] = (double)Pnew[c * cap + i];
  }
  if (io) io[j] = iters[i];
}

template <int NQ>
__global__ void k_sum_parts(const double *parts, int nb, double *out) {
  __shared__ double sh[NQ][256];
  for (int q = 0; q < NQ; q++) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += parts[(size_t)b * NQ + q];
    sh[q][threadIdx.x] = s;
  }
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int q = 0; q < NQ; q++) sh[q][threadIdx.x] += sh[q][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < NQ) out[threadIdx.x] = sh[threadIdx.x][0];
}

template <typename T>
PView<T> pview(pic_ctx *ctx) {
  PView<T> v;
  v.np = ctx->np;
  v.cap = ctx->cap;
  v.cell = ctx->cell;
  v.off = (const T *)ctx->off;
  v.P = (const T *)ctx->P;
  v.Am = (const T *)ctx->Am;
  v.v0 = (const T *)ctx->v0;
  v.w = ctx->w;
  v.sp = ctx->sp;
  v.vbar = (T *)ctx->vbar;
  v.Pnew = (T *)ctx->Pnew;
  v.iters = ctx->iters;
  return v;
}

StepConst base_sc(const pic_ctx *ctx) {
  StepConst sc;
  memset(&sc, 0, sizeof sc);
  sc.dt = ctx->dt;
  sc.kappa = ctx->opt.kappa;
  for (int s = 0; s < PIC_MAX_SPECIES; s++) {
    sc.qs[s] = s < ctx->nspecies ? ctx->qs[s] : 0.0;
    sc.ms[s] = s < ctx->nspecies ? ctx->ms[s] : 1.0;
  }
  return sc;
}

// dispatch on (dim, real type)
#define PIC_DISPATCH(ctx, KCALL)                                   \
  do {                                                             \
    if ((ctx)->rsize == 8) {                                       \
      typedef double RT;                                           \
      if ((ctx)->g.dim == 1) { constexpr int DD = 1; KCALL; }      \
      else if ((ctx)->g.dim == 2) { constexpr int DD = 2; KCALL; } \
      else { constexpr int DD = 3; KCALL; }                        \
    } else {                                                       \
      typedef float RT;                                            \
      if ((ctx)->g.dim == 1) { constexpr int DD = 1; KCALL; }      \
      else if ((ctx)->g.dim == 2) { constexpr int DD = 2; KCALL; } \
      else { constexpr int DD = 3; KCALL; }                        \
    }                                                              \
  } while (0)

}  // namespace

int particles_alloc(pic_ctx *ctx, int64_t n) {
  if (n <= ctx->cap && ctx->cell) return PIC_OK;
  void **bufs[] = {(void **)&ctx->cell, &ctx->off, &ctx->P, (void **)&ctx->w, (void **)&ctx->sp,
                   (void **)&ctx->id, &ctx->Am, &ctx->v0, &ctx->vbar, &ctx->Pnew,
                   (void **)&ctx->iters, (void **)&ctx->u_in, (void **)&ctx->tmp_d,
                   (void **)&ctx->tmp_i, (void **)&ctx->psum};
  for (void **b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  int64_t cap = n > 0 ? n : 1;
  size_t R = (size_t)ctx->rsize;
  size_t nb = (size_t)nblk(cap) + 1;
  CK(cudaMalloc((void **)&ctx->cell, sizeof(int32_t) * 3 * cap));
  CK(cudaMalloc(&ctx->off, R * 3 * cap));
  CK(cudaMalloc(&ctx->P, R * 3 * cap));
  CK(cudaMalloc((void **)&ctx->w, sizeof(double) * cap));
  CK(cudaMalloc((void **)&ctx->sp, sizeof(int32_t) * cap));
  CK(cudaMalloc((void **)&ctx->id, sizeof(int64_t) * cap));
  CK(cudaMalloc(&ctx->Am, R * 3 * cap));
  CK(cudaMalloc(&ctx->v0, R * 3 * cap));
  CK(cudaMalloc(&ctx->vbar, R * 3 * cap));
  CK(cudaMalloc(&ctx->Pnew, R * 3 * cap));
  CK(cudaMalloc((void **)&ctx->iters, sizeof(int32_t) * cap));
  CK(cudaMalloc((void **)&ctx->u_in, sizeof(double) * 3 * cap));
  CK(cudaMalloc((void **)&ctx->tmp_d, sizeof(double) * 7 * cap));
  CK(cudaMalloc((void **)&ctx->tmp_i, sizeof(int32_t) * cap));
  CK(cudaMalloc((void **)&ctx->psum, sizeof(double) * 4 * nb + 64));
  CK(cudaMemsetAsync(ctx->cell, 0, sizeof(int32_t) * 3 * cap, ctx->st));
  CK(cudaMemsetAsync(ctx->off, 0, R * 3 * cap, ctx->st));
  ctx->cap = cap;
  return PIC_OK;
}

int particles_load(pic_ctx *ctx, const int32_t *sp, const double *x, const double *uP,
                   int canonical, const double *w, int on_device) {
  int64_t n = ctx->np, cap = ctx->cap;
  if (n == 0) return PIC_OK;
  const int d = ctx->g.dim;
  const double *dx = x, *du = uP, *dw = w;
  const int32_t *dsp = sp;
  if (!on_device) {
    double *stg = ctx->tmp_d;
    CK(cudaMemcpyAsync(stg, x, sizeof(double) * d * n, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(stg + 3 * cap, uP, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(stg + 6 * cap, w, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
    dx = stg;
    du = stg + 3 * cap;
    dw = stg + 6 * cap;
    if (sp) {
      CK(cudaMemcpyAsync(ctx->tmp_i, sp, sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->st));
      dsp = ctx->tmp_i;
    }
  }
  PGeom pg = pgeom(ctx);
  PIC_DISPATCH(ctx, (k_load<DD, RT><<<nblk(n), kPT, 0, ctx->st>>>(
                         n, cap, dx, du, canonical, dw, dsp, pg, ctx->cell, (RT *)ctx->off,
                         (RT *)ctx->P, ctx->u_in, ctx->w, ctx->sp, ctx->id)));
  KCHECK();
  CK(cudaStreamSynchronize(ctx->st));
  return PIC_OK;
}

int particles_form_P(pic_ctx *ctx) {
  if (ctx->np == 0) return PIC_OK;
  PGeom pg = pgeom(ctx);
  StepConst sc = base_sc(ctx);
  PIC_DISPATCH(ctx, (k_form_P<DD, RT><<<nblk(ctx->np), kPT, 0, ctx->st>>>(
                         pview<RT>(ctx), (RT *)ctx->P, ctx->u_in, ctx->A_real, pg, sc)));
  KCHECK();
  return PIC_OK;
}

int particles_point_deposit(pic_ctx *ctx, double *rho, double *J) {
  if (ctx->np == 0) return PIC_OK;
  PGeom pg = pgeom(ctx);
  StepConst sc = base_sc(ctx);
  PIC_DISPATCH(ctx, (k_point_deposit<DD, RT><<<nblk(ctx->np), kPT, 0, ctx->st>>>(
                         pview<RT>(ctx), ctx->A_real, pg, sc, rho, J)));
  KCHECK();
  return PIC_OK;
}

int particles_step_start(pic_ctx *ctx) {
  if (ctx->np == 0) return PIC_OK;
  PGeom pg = pgeom(ctx);
  StepConst sc = base_sc(ctx);
  PIC_DISPATCH(ctx, (k_step_start<DD, RT><<<nblk(ctx->np), kPT, 0, ctx->st>>>(
                         pview<RT>(ctx), (RT *)ctx->Am, (RT *)ctx->v0, ctx->A_real, pg, sc)));
  KCHECK();
  return PIC_OK;
}

int particles_map(pic_ctx *ctx, const StepConst &sc_in, int final_pass, double *work_sum,
                  double *chain_sum, EvalCounters *cnt) {
  EvalCounters zero = {0u, 0, 0ull};
  CK(cudaMemcpyAsync(ctx->cnt_dev, &zero, sizeof zero, cudaMemcpyHostToDevice, ctx->st));
  int nb = nblk(ctx->np);
  double *res = ctx->red_host + 16;  // work, chain, inner iterations, pieces
  if (ctx->np > 0) {
    PGeom pg = pgeom(ctx);
    StepConst sc = sc_in;
    CK(cudaEventRecord(ctx->ev0, ctx->st));
    PIC_DISPATCH(ctx, (k_map<DD, RT><<<nb, kPT, 0, ctx->st>>>(
                           pview<RT>(ctx), (const RT *)ctx->nodes, (const RT *)ctx->nodes_u,
                           ctx->Jorb, pg, sc, final_pass, ctx->cnt_dev, ctx->psum)));
    KCHECK();
    CK(cudaEventRecord(ctx->ev1, ctx->st));
    k_sum_parts<4><<<1, 256, 0, ctx->st>>>(ctx->psum, nb, ctx->psum + (size_t)4 * nb);
    KCHECK();
    CK(cudaMemcpyAsync(res, ctx->psum + (size_t)4 * nb, sizeof(double) * 4,
                       cudaMemcpyDeviceToHost, ctx->st));
  } else {
    res[0] = res[1] = res[2] = res[3] = 0.0;
  }
  CK(cudaMemcpyAsync(ctx->cnt_host, ctx->cnt_dev, sizeof(EvalCounters), cudaMemcpyDeviceToHost,
                     ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (ctx->np > 0) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    ctx->map_ms += ms;
    ctx->map_launches++;
  }
  *cnt = *ctx->cnt_host;
  cnt->inner_sum = (unsigned long long)(res[2] + 0.5);
  ctx->pushes += ctx->np;
  ctx->inner_iters += (long long)(res[2] + 0.5);
  ctx->pieces += (long long)(res[3] + 0.5);
  if (work_sum) *work_sum = res[0];
  if (chain_sum) *chain_sum = res[1];
  return PIC_OK;
}

int particles_commit(pic_ctx *ctx) {
  if (ctx->np == 0) return PIC_OK;
  PGeom pg = pgeom(ctx);
  PIC_DISPATCH(ctx, (k_commit<DD, RT><<<nblk(ctx->np), kPT, 0, ctx->st>>>(
                         ctx->np, ctx->cap, ctx->cell, (RT *)ctx->off, (RT *)ctx->P,
                         (const RT *)ctx->vbar, (const RT *)ctx->Pnew, pg, ctx->dt)));
  KCHECK();
  return PIC_OK;
}

int particles_kinetic(pic_ctx *ctx, double *K) {
  if (ctx->np == 0) { *K = 0.0; return PIC_OK; }
  PGeom pg = pgeom(ctx);
  StepConst sc = base_sc(ctx);
  int nb = nblk(ctx->np);
  PIC_DISPATCH(ctx, (k_kinetic<DD, RT><<<nb, kPT, 0, ctx->st>>>(pview<RT>(ctx), ctx->A_real,
                                                                  pg, sc, ctx->psum)));
  KCHECK();
  k_sum_parts<1><<<1, 256, 0, ctx->st>>>(ctx->psum, nb, ctx->psum + nb);
  KCHECK();
  CK(cudaMemcpyAsync(ctx->red_host + 24, ctx->psum + nb, sizeof(double), cudaMemcpyDeviceToHost,
                     ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  *K = ctx->red_host[24];
  return PIC_OK;
}

int particles_export(pic_ctx *ctx, double *x, double *P, double *w, int32_t *sp, int on_device) {
  int64_t n = ctx->np;
  if (n == 0) return PIC_OK;
  const int d = ctx->g.dim;
  double *dx = x, *dP = P, *dw = w;
  int32_t *dsp = sp;
  if (!on_device) {
    dx = x ? ctx->tmp_d : nullptr;
    dP = P ? ctx->tmp_d + 3 * ctx->cap : nullptr;
    dw = w ? ctx->tmp_d + 6 * ctx->cap : nullptr;
    dsp = sp ? ctx->tmp_i : nullptr;
  }
  PGeom pg = pgeom(ctx);
  PIC_DISPATCH(ctx, (k_export<DD, RT><<<nblk(n), kPT, 0, ctx->st>>>(pview<RT>(ctx), ctx->id, pg,
                                                                      dx, dP, dw, dsp)));
  KCHECK();
  if (!on_device) {
    if (x) CK(cudaMemcpyAsync(x, dx, sizeof(double) * d * n, cudaMemcpyDeviceToHost, ctx->st));
    if (P) CK(cudaMemcpyAsync(P, dP, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->st));
    if (w) CK(cudaMemcpyAsync(w, dw, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->st));
    if (sp) CK(cudaMemcpyAsync(sp, dsp, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, ctx->st));
  }
  CK(cudaStreamSynchronize(ctx->st));
  return PIC_OK;
}

int particles_export_eval(pic_ctx *ctx, double *vbar, double *Pnew, int32_t *iters,
                          int on_device) {
  int64_t n = ctx->np;
  if (n == 0) return PIC_OK;
  double *dv = vbar, *dP = Pnew;
  int32_t *di = iters;
  if (!on_device) {
    dv = vbar ? ctx->tmp_d : nullptr;
    dP = Pnew ? ctx->tmp_d + 3 * ctx->cap : nullptr;
    di = iters ? ctx->tmp_i : nullptr;
  }
  if (ctx->rsize == 8)
    k_export_eval<double><<<nblk(n), kPT, 0, ctx->st>>>(n, ctx->cap, ctx->id,
                                                        (const double *)ctx->vbar,
                                                        (const double *)ctx->Pnew, ctx->iters, dv,
                                                        dP, di);
  else
    k_export_eval<float><<<nblk(n), kPT, 0, ctx->st>>>(n, ctx->cap, ctx->id,
                                                       (const float *)ctx->vbar,
                                                       (const float *)ctx->Pnew, ctx->iters, dv,
                                                       dP, di);
  KCHECK();
  if (!on_device) {
    if (vbar) CK(cudaMemcpyAsync(vbar, dv, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->st));
    if (Pnew) CK(cudaMemcpyAsync(Pnew, dP, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->st));
    if (iters) CK(cudaMemcpyAsync(iters, di, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, ctx->st));
  }
  CK(cudaStreamSynchronize(ctx->st));
  return PIC_OK;
}

int particles_sort(pic_ctx *ctx) {
  (void)ctx;
  return PIC_OK;
}
