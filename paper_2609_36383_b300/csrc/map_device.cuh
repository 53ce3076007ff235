// map_device.cuh -- device code of the particle map: geometry and constants,
// the knot-split orbit walk, the orbit gather and deposit functors, the GM-HC
// push, the convergence-triggered refinement retry, and map_block(), the
// per-thread body of the map kernel.  Included by particle.cu (one problem per launch) and
// batch.cu (many independent problems per launch).
//
// One thread owns one particle and runs its inner Picard iteration (Sec. 4.5)
// to convergence:
//   orbit x(s) = x^n + s dt vbar (Eq. rel-orbit), split at every crossed knot
//   of the B-spline (half-integer node coordinates for the quadratic S_2,
//   also the nodes for the linear S_1 of Sec. 5.3), Gauss-Legendre
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
#pragma once

#include "dual.cuh"
#include "pic_internal.cuh"

#include <cmath>
#include <type_traits>

namespace {

constexpr int kPT = 128;     // particle kernel block size
constexpr int kMaxPieces = 16;

struct PGeom {
  int n[3], mask[3];
  int Ng, n0, n01;
  int order;  // B-spline degree of the particle shape: 2, or 1 (Sec. 5.3)
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
  p.order = ctx->opt.order;
  p.n0 = ctx->g.n[0];
  p.n01 = ctx->g.n[0] * ctx->g.n[1];
  p.inv_dV = 1.0 / ctx->g.dV;
  return p;
}

inline int nblk(int64_t n) { return (int)((n + kPT - 1) / kPT); }

// Constants of the particle map in the particle real type, so that the FP32
// instance does no FP64 conversion inside its loops (the FP64 pipe of the
// B300 is 1/64 of the FP32 one).
template <typename T>
struct KConst {
  T dt, kappa, tau_r, tau_a, inv_dV;
  T inv_dx[3];
  T gl_t[PIC_MAX_GL], gl_w[PIC_MAX_GL];
  int ngl, inner_max, warm;
  int order;       // shape degree (2, or 1)
  int refine_max;  // convergence-triggered refinement depth (0 = off)
  double qs[PIC_MAX_SPECIES], ms[PIC_MAX_SPECIES];
  T qT[PIC_MAX_SPECIES], mT[PIC_MAX_SPECIES];  // the same in the particle real type
};

// Mesh scales of one problem in the particle real type, kept apart from
// KConst so that a kernel serving several problems can set them per CTA
// without copying KConst (and its indexed tables) out of parameter space.
template <typename T>
struct MapScale {
  T inv_dx[3];
  T inv_dV;
};

template <typename T>
KConst<T> kconst(const StepConst &sc, const PGeom &pg) {
  KConst<T> k;
  k.dt = (T)sc.dt;
  k.kappa = (T)sc.kappa;
  k.tau_r = (T)sc.tau_r;
  k.tau_a = (T)sc.tau_a;
  k.inv_dV = (T)pg.inv_dV;
  for (int l = 0; l < 3; l++) k.inv_dx[l] = (T)pg.inv_dx[l];
  for (int q = 0; q < PIC_MAX_GL; q++) {
    k.gl_t[q] = (T)sc.gl_t[q];
    k.gl_w[q] = (T)sc.gl_w[q];
  }
  k.ngl = sc.ngl;
  k.inner_max = sc.inner_max;
  k.warm = sc.warm;
  k.order = sc.order;
  k.refine_max = sc.refine_max;
  for (int s = 0; s < PIC_MAX_SPECIES; s++) {
    k.qs[s] = sc.qs[s];
    k.ms[s] = sc.ms[s];
    k.qT[s] = (T)sc.qs[s];
    k.mT[s] = (T)sc.ms[s];
  }
  return k;
}

// Exact widening of a deposit contribution to FP64 for the global atomics.
// For FP32 the conversion is done with integer operations (sign, exponent
// rebias by 1023 - 127 = 896, mantissa shift by 29) so that it does not
// occupy the narrow FP64 pipe; FP32 subnormals (< 1.2e-38) flush to zero,
// and the FP32 infinities and NaNs (exponent 255) stay infinities and NaNs.
// Deposit of one contribution into the FP64 current J (3 Ng values); a Dual
// contribution also deposits its tangent into the array that follows J.
__device__ __forceinline__ void dep_add(double *J, size_t idx, size_t, double v) {
  atomicAdd(J + idx, v);
}
__device__ __forceinline__ double widen(float v);
__device__ __forceinline__ void dep_add(double *J, size_t idx, size_t, float v) {
  atomicAdd(J + idx, widen(v));
}
__device__ __forceinline__ void dep_add(double *J, size_t idx, size_t span, const Dual &v) {
  atomicAdd(J + idx, v.v);
  atomicAdd(J + span + idx, v.d);
}

__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  if (e == 0xffu)
    return __hiloint2double((int)((u & 0x80000000u) | 0x7ff00000u | ((u >> 3) & 0x000fffffu)),
                            (int)(u << 29));
  const unsigned hi = (u & 0x80000000u) | ((((u >> 3) & 0x0fffffffu)) + (896u << 20));
  const unsigned lo = u << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// B-spline weights of the three nodes b-1, b, b+1 for t = u - b in
// [-1/2, 1/2], and their derivatives with respect to u.  Degree 2 (the
// quadratic S_2, knots at half-integers); degree 1 (the hat S_1 of Sec. 5.3,
// knots on the nodes), where `pos` says on which side of node b the
// knot-split piece lies (t >= 0), so that a quadrature point that rounding
// puts on the wrong side of the knot still takes its piece's polynomial.
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
__device__ __forceinline__ void lspline(T t, bool pos, T S[3], T dS[3]) {
  S[0] = pos ? T(0) : -t;
  S[1] = pos ? T(1) - t : T(1) + t;
  S[2] = pos ? t : T(0);
  dS[0] = pos ? T(0) : T(-1);
  dS[1] = pos ? T(-1) : T(1);
  dS[2] = pos ? T(1) : T(0);
}

template <typename T>
__device__ __forceinline__ void qspline_val(T t, T S[3]) {
  T a = T(0.5) - t, b = T(0.5) + t;
  S[0] = T(0.5) * a * a;
  S[1] = T(0.75) - t * t;
  S[2] = T(0.5) * b * b;
}

// point weights of the particle shape of degree `order`
template <typename T>
__device__ __forceinline__ void spline_val(int order, T t, T S[3]) {
  if (order == 1) {
    S[0] = t < T(0) ? -t : T(0);
    S[1] = T(1) - fabs(t);
    S[2] = t > T(0) ? t : T(0);
  } else {
    qspline_val<T>(t, S);
  }
}

template <int D>
__device__ __forceinline__ int node_index(const PGeom &pg, const int cell[3], const int base[3],
                                          const int o[3]) {
  int g = (cell[0] + base[0] + o[0]) & pg.mask[0];
  if (D > 1) g += pg.n0 * ((cell[1] + base[1] + o[1]) & pg.mask[1]);
  if (D > 2) g += pg.n01 * ((cell[2] + base[2] + o[2]) & pg.mask[2]);
  return g;
}

// Wrapped node coordinates of the 3 nodes around base along each active
// dimension, pre-scaled by the dimension's stride: node (ox, oy, oz) is
// gx[ox] + gy[oy] + gz[oz].
template <int D>
struct NodeRows {
  int gx[3], gy[3], gz[3];
  __device__ __forceinline__ NodeRows(const PGeom &pg, const int cell[3], const int base[3]) {
#pragma unroll
    for (int o = 0; o < 3; o++) {
      gx[o] = (cell[0] + base[0] + o - 1) & pg.mask[0];
      gy[o] = D > 1 ? pg.n0 * ((cell[1] + base[1] + o - 1) & pg.mask[1]) : 0;
      gz[o] = D > 2 ? pg.n01 * ((cell[2] + base[2] + o - 1) & pg.mask[2]) : 0;
    }
  }
  __device__ __forceinline__ int at(int ox, int oy, int oz) const {
    return gx[ox] + (D > 1 ? gy[oy] : 0) + (D > 2 ? gz[oz] : 0);
  }
};

// Walks the knot-split pieces of the straight orbit u(s) = off + s del,
// s in [0, 1], calling f(base, sa, sb) on each piece, where base is the node
// (relative to the particle's cell) nearest to u inside the piece.  Pieces
// end where the orbit crosses a half-integer coordinate (the knots of S_2,
// where the nearest node also changes); for degree-one shapes (order 1) also
// where it crosses a node (the knots of S_1).  Returns false if the orbit has
// more pieces than kMaxPieces.
template <int D, typename T, typename F>
__device__ __forceinline__ bool walk_orbit(const T off[3], const T del[3], F &f, int order) {
  T d0[3], stp[3], nxt[3];
  int kc[3];
  const T h = order == 1 ? T(0.5) : T(1);  // spacing of the split points
#pragma unroll
  for (int l = 0; l < D; l++) {
    kc[l] = 0;
    if (del[l] == T(0)) {
      nxt[l] = T(2);
      stp[l] = T(0);
      d0[l] = T(0);
      continue;
    }
    if (del[l] > T(0))
      d0[l] = (order == 1 && off[l] < T(0)) ? -off[l] : T(0.5) - off[l];
    else
      d0[l] = (order == 1 && off[l] > T(0)) ? off[l] : off[l] + T(0.5);
    if (d0[l] <= T(0)) d0[l] = h;
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
        nxt[l] = (d0[l] + T(kc[l]) * h) * stp[l];
      }
    sa = sb;
  }
  return false;
}

// Node records: [grad phi^{1/2} (D), A^n (3), A^{n+1} (3)] padded to a
// multiple of four reals, so one record is read with 16-byte vector loads.
template <int D>
struct Rec {
  static constexpr int NVP = (D + 6 + 3) / 4 * 4;
};

template <int N>
__device__ __forceinline__ void load_rec(const double *__restrict__ p, double (&o)[N]) {
#pragma unroll
  for (int k = 0; k < N / 2; k++) {
    double2 v = __ldg(reinterpret_cast<const double2 *>(p) + k);
    o[2 * k] = v.x;
    o[2 * k + 1] = v.y;
  }
}

template <int N>
__device__ __forceinline__ void load_rec(const Dual *__restrict__ p, Dual (&o)[N]) {
#pragma unroll
  for (int k = 0; k < N; k++) {
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p) + k);
    o[k] = Dual(v.x, v.y);
  }
}

template <int N>
__device__ __forceinline__ void load_rec(const float *__restrict__ p, float (&o)[N]) {
#pragma unroll
  for (int k = 0; k < N / 4; k++) {
    float4 v = __ldg(reinterpret_cast<const float4 *>(p) + k);
    o[4 * k] = v.x;
    o[4 * k + 1] = v.y;
    o[4 * k + 2] = v.z;
    o[4 * k + 3] = v.w;
  }
}

// Orbit integrals over one knot-split piece [sa, sb], accumulated over its
// Gauss-Legendre points for the 3^D nodes around the piece's base node:
//   Sb[k]    = int S_k(x(s)) ds
//   Wd[j][k] = int d S_k / d u_j ds        (node units; scaled by 1/dx_j later)
//   W1[j][k] = int s d S_k / d u_j ds
// With A(s) = (1-s) A^n + s A^{n+1} (Eq. A-g-s) the discrete gradient of
// Eq. D-def is then sum_k A^n_k Wd_k + (A^{n+1}_k - A^n_k) W1_k.
template <int D, typename T>
struct PieceAcc {
  static constexpr int NN = D == 1 ? 3 : (D == 2 ? 9 : 27);
  T Sb[NN];
  T Wd[D][NN];
  T W1[D][NN];
};

// One Gauss-Legendre point (s, weight wt) of a piece's orbit integrals;
// FIRST assigns the point's terms (the piece's first point) instead of
// adding them, so the accumulators need no clearing.
template <bool FIRST, typename T>
__device__ __forceinline__ void acc_put(T &x, T v) {
  if (FIRST) x = v;
  else x += v;
}

template <int D, typename T, bool DERIV, bool FIRST>
__device__ __forceinline__ void piece_point(const T t0[3], const bool pos[3], bool lin,
                                            const T del[3], T s, T wt, PieceAcc<D, T> &pa) {
  T S[3][3], dS[3][3];
#pragma unroll
  for (int l = 0; l < D; l++) {
    if (lin) lspline<T>(t0[l] + s * del[l], pos[l], S[l], dS[l]);
    else qspline<T>(t0[l] + s * del[l], S[l], dS[l]);
  }
  if (D == 1) {
#pragma unroll
    for (int i = 0; i < 3; i++) {
      acc_put<FIRST>(pa.Sb[i], wt * S[0][i]);
      if (DERIV) {
        T b = wt * dS[0][i];
        acc_put<FIRST>(pa.Wd[0][i], b);
        acc_put<FIRST>(pa.W1[0][i], s * b);
      }
    }
  } else if (D == 2) {
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const T a = wt * S[0][i];
      const T b = wt * dS[0][i];
      const T c = s * a, e = s * b;
#pragma unroll
      for (int j = 0; j < 3; j++) {
        const int k = i + 3 * j;
        acc_put<FIRST>(pa.Sb[k], a * S[1][j]);
        if (DERIV) {
          acc_put<FIRST>(pa.Wd[0][k], b * S[1][j]);
          acc_put<FIRST>(pa.W1[0][k], e * S[1][j]);
          acc_put<FIRST>(pa.Wd[D > 1 ? 1 : 0][k], a * dS[1][j]);
          acc_put<FIRST>(pa.W1[D > 1 ? 1 : 0][k], c * dS[1][j]);
        }
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int j = 0; j < 3; j++) {
        const T ab = wt * S[0][i] * S[1][j];
        const T dab = wt * dS[0][i] * S[1][j];
        const T adb = wt * S[0][i] * dS[1][j];
#pragma unroll
        for (int l = 0; l < 3; l++) {
          const int k = i + 3 * (j + 3 * l);
          acc_put<FIRST>(pa.Sb[k], ab * S[2][l]);
          if (DERIV) {
            const T d0 = dab * S[2][l], d1 = adb * S[2][l], d2 = ab * dS[2][l];
            acc_put<FIRST>(pa.Wd[0][k], d0);
            acc_put<FIRST>(pa.W1[0][k], s * d0);
            acc_put<FIRST>(pa.Wd[D > 1 ? 1 : 0][k], d1);
            acc_put<FIRST>(pa.W1[D > 1 ? 1 : 0][k], s * d1);
            acc_put<FIRST>(pa.Wd[D > 2 ? 2 : 0][k], d2);
            acc_put<FIRST>(pa.W1[D > 2 ? 2 : 0][k], s * d2);
          }
        }
      }
  }
}

// The orbit integrals of one piece over its kc.ngl Gauss-Legendre points.
template <int D, typename T, bool DERIV>
__device__ __forceinline__ void accumulate_piece(const KConst<T> &kc, const T off[3],
                                                 const T del[3], const int base[3], T sa, T sb,
                                                 PieceAcc<D, T> &pa, int order) {
  const T len = sb - sa;
  T t0[3];
  bool pos[3] = {false, false, false};
  const bool lin = order == 1;
#pragma unroll
  for (int l = 0; l < D; l++) {
    t0[l] = off[l] - T(base[l]);
    if (lin) pos[l] = t0[l] + T(0.5) * (sa + sb) * del[l] >= T(0);
  }
  if constexpr (!std::is_same<T, float>::value) {
    // FP64 (and dual numbers): cleared accumulators and a rolled point loop,
    // the smaller code for a kernel bound by the FP64 pipe
    constexpr int NN = PieceAcc<D, T>::NN;
#pragma unroll
    for (int k = 0; k < NN; k++) {
      pa.Sb[k] = T(0);
#pragma unroll
      for (int j = 0; j < D; j++) pa.Wd[j][k] = pa.W1[j][k] = T(0);
    }
#pragma unroll 1
    for (int qp = 0; qp < kc.ngl; qp++)
      piece_point<D, T, DERIV, false>(t0, pos, lin, del, sa + len * kc.gl_t[qp],
                                      len * kc.gl_w[qp], pa);
    return;
  }
  // FP32: the first point assigns (no clearing); without derivatives and
  // with the default rule the point loop is unrolled
  piece_point<D, T, DERIV, true>(t0, pos, lin, del, sa + len * kc.gl_t[0], len * kc.gl_w[0], pa);
  if (!DERIV && kc.ngl == D + 1) {
#pragma unroll
    for (int qp = 1; qp < D + 1; qp++)
      piece_point<D, T, DERIV, false>(t0, pos, lin, del, sa + len * kc.gl_t[qp],
                                      len * kc.gl_w[qp], pa);
    return;
  }
#pragma unroll 1
  for (int qp = 1; qp < kc.ngl; qp++)
    piece_point<D, T, DERIV, false>(t0, pos, lin, del, sa + len * kc.gl_t[qp], len * kc.gl_w[qp],
                                    pa);
}

// 3D: the same orbit integrals for the 9 nodes (ox, oy) of one z-slab oz of
// the 27-node stencil, so that the accumulators of a slab (9 x 7 values) fit
// in registers; the caller loops over the three slabs and contracts each.
template <typename T, bool DERIV>
__device__ __forceinline__ void accumulate_slab(const KConst<T> &kc, const T off[3],
                                                const T del[3], const int base[3], T sa, T sb,
                                                int oz, PieceAcc<2, T> &pa, T (&Wz)[9],
                                                T (&W1z)[9], int order) {
#pragma unroll
  for (int k = 0; k < 9; k++) {
    pa.Sb[k] = T(0);
    pa.Wd[0][k] = pa.W1[0][k] = pa.Wd[1][k] = pa.W1[1][k] = T(0);
    Wz[k] = W1z[k] = T(0);
  }
  const T len = sb - sa;
  T t0[3];
  bool pos[3] = {false, false, false};
  const bool lin = order == 1;
#pragma unroll
  for (int l = 0; l < 3; l++) {
    t0[l] = off[l] - T(base[l]);
    if (lin) pos[l] = t0[l] + T(0.5) * (sa + sb) * del[l] >= T(0);
  }
#pragma unroll 1
  for (int qp = 0; qp < kc.ngl; qp++) {
    const T s = sa + len * kc.gl_t[qp];
    const T wt = len * kc.gl_w[qp];
    T S[3][3], dS[3][3];
#pragma unroll
    for (int l = 0; l < 3; l++) {
      if (lin) lspline<T>(t0[l] + s * del[l], pos[l], S[l], dS[l]);
      else qspline<T>(t0[l] + s * del[l], S[l], dS[l]);
    }
    const T wz = wt * S[2][oz], wdz = wt * dS[2][oz];
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const T a = wz * S[0][i], b = wz * dS[0][i], az = wdz * S[0][i];
#pragma unroll
      for (int j = 0; j < 3; j++) {
        const int k = i + 3 * j;
        pa.Sb[k] += a * S[1][j];
        if (DERIV) {
          const T d0 = b * S[1][j], d1 = a * dS[1][j], d2 = az * S[1][j];
          pa.Wd[0][k] += d0;
          pa.W1[0][k] += s * d0;
          pa.Wd[1][k] += d1;
          pa.W1[1][k] += s * d1;
          Wz[k] += d2;
          W1z[k] += s * d2;
        }
      }
    }
  }
}

// One node's terms of the discrete gradient (node units), for the NC
// columns j with orbit integrals wd[j] = int dS/du_j and w1[j] = int s dS/du_j:
//   Dm[c][j] += A^n_c wd[j] + (A^{n+1}_c - A^n_c) w1[j]
// evaluated as A^n_c (wd[j] - w1[j]) + A^{n+1}_c w1[j], two FMAs per term
// (r: the node record, A^n at r[D + c], A^{n+1} at r[D + 3 + c]).  On a
// substep (SUB) the potential is A^n + (ta + s tsp) (A^{n+1} - A^n).
template <int NC, int D, typename T, bool SUB>
__device__ __forceinline__ void dgrad_node(T (&Dm)[3][3], const T *r, const T (&wd)[NC],
                                           const T (&w1)[NC], T ta, T tsp) {
  if (SUB) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      T An = r[D + c], dA = r[D + 3 + c] - An;
      An += ta * dA;
      dA *= tsp;
#pragma unroll
      for (int j = 0; j < NC; j++) Dm[c][j] += An * wd[j] + dA * w1[j];
    }
    return;
  }
  T wm[NC];
#pragma unroll
  for (int j = 0; j < NC; j++) wm[j] = wd[j] - w1[j];
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int j = 0; j < NC; j++) {
      Dm[c][j] += r[D + c] * wm[j];
      Dm[c][j] += r[D + 3 + c] * w1[j];
    }
}

// Inner-iteration gather: grad phi-bar (Eq. orbit-gather-general with
// G = grad phi^{1/2}) and the discrete gradient D (3 x D, node units until
// the caller scales column j by 1/dx_j).
// SUB: the orbit covers the part [ta, ta + tsp] of the field step (a
// substep of convergence-triggered refinement), over which the potential is
// A^n + (ta + s tsp) (A^{n+1} - A^n) (Eq. A-g-s); otherwise ta = 0, tsp = 1.
template <int D, typename T, bool SUB = false>
struct GatherOrbit {
  const T *__restrict__ nodes;
  const PGeom *pg;
  const KConst<T> *kc;
  int cell[3];
  T off[3], del[3];
  T gphi[3];
  T Dm[3][3];
  T ta, tsp;
  int order;  // shape degree (a literal 2 on the common path, folded by the compiler)
  int pieces;
  __device__ __forceinline__ void operator()(const int base[3], T sa, T sb) {
    constexpr int NVP = Rec<D>::NVP;
    pieces++;
    const NodeRows<D> nr(*pg, cell, base);
    if (D == 3) {
#pragma unroll 1
      for (int oz = 0; oz < 3; oz++) {
        PieceAcc<2, T> pa;
        T Wz[9], W1z[9];
        accumulate_slab<T, true>(*kc, off, del, base, sa, sb, oz, pa, Wz, W1z, order);
#pragma unroll
        for (int oy = 0; oy < 3; oy++)
#pragma unroll
          for (int ox = 0; ox < 3; ox++) {
            const int k = ox + 3 * oy;
            const int g = nr.at(ox, oy, oz);
            T r[NVP];
            load_rec<NVP>(nodes + (size_t)g * NVP, r);
#pragma unroll
            for (int c = 0; c < D; c++) gphi[c] += r[c] * pa.Sb[k];
            const T wd[3] = {pa.Wd[0][k], pa.Wd[1][k], Wz[k]};
            const T w1[3] = {pa.W1[0][k], pa.W1[1][k], W1z[k]};
            dgrad_node<3, D, T, SUB>(Dm, r, wd, w1, ta, tsp);
          }
      }
      return;
    }
    PieceAcc<D, T> pa;
    accumulate_piece<D, T, true>(*kc, off, del, base, sa, sb, pa, order);
#pragma unroll
    for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
#pragma unroll
      for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
#pragma unroll
        for (int ox = 0; ox < 3; ox++) {
          const int k = ox + 3 * (oy + 3 * oz);
          const int g = nr.at(ox, oy, oz);
          T r[NVP];
          load_rec<NVP>(nodes + (size_t)g * NVP, r);
#pragma unroll
          for (int c = 0; c < D; c++) gphi[c] += r[c] * pa.Sb[k];
          T wd[D], w1[D];
#pragma unroll
          for (int j = 0; j < D; j++) {
            wd[j] = pa.Wd[j][k];
            w1[j] = pa.W1[j][k];
          }
          dgrad_node<D, D, T, SUB>(Dm, r, wd, w1, ta, tsp);
        }
  }
};

// Warp deposit window of the FP32 path: the nodes within [-2, 3] x [-2, 2]
// (1D: [-2, 3]) of the cell of the warp's first particle, 3 components each.
// Every lane accumulates into its own column of the window in shared memory
// (element e of lane l at (e * 32 + l): bank = lane, no conflicts and no
// shared atomics); afterwards the warp sums the 32 columns and issues one
// FP64 global atomic per touched entry.  Contributions outside the window go
// straight to global atomics.  With particles sorted by cell a warp holds one
// or two neighbouring cells, so nearly all contributions land in the window.
template <int D>
struct WarpWin {
  static constexpr bool kOn = D <= 2;
  static constexpr int LO0 = -2, N0 = 6, LO1 = -2, N1 = D > 1 ? 5 : 1;
  static constexpr int NE = 3 * N0 * N1;  // entries per lane
};

__device__ __forceinline__ int wrap_rel(int v, int n) {  // into [-n/2, n/2)
  v &= n - 1;
  return v >= n / 2 ? v - n : v;
}

// Orbit deposit of q vbar Sbar / dV (Eq. orbit-current-energy); on the final
// pass also the gathers behind the work and chain-rule diagnostics.
template <int D, typename T, bool FINAL, bool SUB = false>
struct DepositOrbit {
  const T *__restrict__ nodes;
  const T *__restrict__ nodes_u;
  double *__restrict__ J;
  const PGeom *pg;
  const KConst<T> *kc;
  int cell[3];
  T off[3], del[3];
  T qv[3];  // q vbar / dV (times the substep's share of the step)
  T gphi[3], Ubar[3], Dm[3][3];
  T ta, tsp;  // substep times, as in GatherOrbit
  int order;
  int pieces;
  T *win;      // this lane's column of the warp window (stride 32), or null
  int ref[3];  // the window's reference cell
  __device__ __forceinline__ void operator()(const int base[3], T sa, T sb) {
    constexpr int NVP = Rec<D>::NVP;
    pieces++;
    const NodeRows<D> nr(*pg, cell, base);
    if (D == 3) {
#pragma unroll 1
      for (int oz = 0; oz < 3; oz++) {
        PieceAcc<2, T> pa;
        T Wz[9], W1z[9];
        accumulate_slab<T, FINAL>(*kc, off, del, base, sa, sb, oz, pa, Wz, W1z, order);
#pragma unroll
        for (int oy = 0; oy < 3; oy++)
#pragma unroll
          for (int ox = 0; ox < 3; ox++) {
            const int k = ox + 3 * oy;
            const int g = nr.at(ox, oy, oz);
            if (FINAL) {
              T r[NVP], u[4];
              load_rec<NVP>(nodes + (size_t)g * NVP, r);
              load_rec<4>(nodes_u + (size_t)g * 4, u);
#pragma unroll
              for (int c = 0; c < D; c++) gphi[c] += r[c] * pa.Sb[k];
#pragma unroll
              for (int c = 0; c < 3; c++) Ubar[c] += u[c] * pa.Sb[k];
              const T wd[3] = {pa.Wd[0][k], pa.Wd[1][k], Wz[k]};
              const T w1[3] = {pa.W1[0][k], pa.W1[1][k], W1z[k]};
              dgrad_node<3, D, T, SUB>(Dm, r, wd, w1, ta, tsp);
            }
#pragma unroll
            for (int c = 0; c < 3; c++)
              dep_add(J, (size_t)c * pg->Ng + g, 3 * (size_t)pg->Ng, qv[c] * pa.Sb[k]);
          }
      }
      return;
    }
    PieceAcc<D, T> pa;
    accumulate_piece<D, T, FINAL>(*kc, off, del, base, sa, sb, pa, order);
    if (FINAL) {
#pragma unroll
      for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
#pragma unroll
        for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
#pragma unroll
          for (int ox = 0; ox < 3; ox++) {
            const int k = ox + 3 * (oy + 3 * oz);
            const int g = nr.at(ox, oy, oz);
            T r[NVP], u[4];
            load_rec<NVP>(nodes + (size_t)g * NVP, r);
            load_rec<4>(nodes_u + (size_t)g * 4, u);
#pragma unroll
            for (int c = 0; c < D; c++) gphi[c] += r[c] * pa.Sb[k];
#pragma unroll
            for (int c = 0; c < 3; c++) Ubar[c] += u[c] * pa.Sb[k];
            T wd[D], w1[D];
#pragma unroll
            for (int j = 0; j < D; j++) {
              wd[j] = pa.Wd[j][k];
              w1[j] = pa.W1[j][k];
            }
            dgrad_node<D, D, T, SUB>(Dm, r, wd, w1, ta, tsp);
          }
    }
    // window coordinates of the piece's base node (relative to ref)
    int wx = -1, wy = -1;
    if (WarpWin<D>::kOn && win) {
      wx = wrap_rel(cell[0] + base[0] - ref[0], pg->n[0]) - 1 - WarpWin<D>::LO0;
      wy = D > 1 ? wrap_rel(cell[1] + base[1] - ref[1], pg->n[1]) - 1 - WarpWin<D>::LO1 : 0;
    }
    if (WarpWin<D>::kOn && win && wx >= 0 && wx + 2 < WarpWin<D>::N0 && wy >= 0 &&
        wy + (D > 1 ? 2 : 0) < WarpWin<D>::N1) {
      // the piece's whole stencil lies in the window: fixed offsets from one base
      T *w0 = win + (size_t)3 * (wx + WarpWin<D>::N0 * wy) * 32;
#pragma unroll
      for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
#pragma unroll
        for (int ox = 0; ox < 3; ox++) {
          const int k = ox + 3 * oy;
#pragma unroll
          for (int c = 0; c < 3; c++)
            w0[(3 * (ox + WarpWin<D>::N0 * oy) + c) * 32] += qv[c] * pa.Sb[k];
        }
      return;
    }
#pragma unroll
    for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
#pragma unroll
      for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
#pragma unroll
        for (int ox = 0; ox < 3; ox++) {
          const int k = ox + 3 * (oy + 3 * oz);
          const int g = nr.at(ox, oy, oz);
          int e = -1;
          if (WarpWin<D>::kOn && win) {
            const int rx = wx + ox, ry = wy + (D > 1 ? oy : 0);
            if (rx >= 0 && rx < WarpWin<D>::N0 && ry >= 0 && ry < WarpWin<D>::N1)
              e = 3 * (rx + WarpWin<D>::N0 * ry);
          }
#pragma unroll
          for (int c = 0; c < 3; c++) {
            const T v = qv[c] * pa.Sb[k];
            if (e >= 0) win[(e + c) * 32] += v;
            else dep_add(J, (size_t)c * pg->Ng + g, 3 * (size_t)pg->Ng, v);
          }
        }
  }
};

// A^{n+1}_h at u = off + del (node coordinates relative to the cell) from the
// node records (Eq. mesh-interpolant)
template <int D, typename T>
__device__ __forceinline__ void interp_A1(const PGeom &pg, const int cell[3], const T u[3],
                                          const T *__restrict__ nodes, T out[3], int order) {
  constexpr int NVP = Rec<D>::NVP;
  int base[3] = {0, 0, 0};
  T Sw[3][3];
#pragma unroll
  for (int l = 0; l < D; l++) {
    base[l] = (int)floor(u[l] + T(0.5));
    spline_val<T>(order, u[l] - T(base[l]), Sw[l]);
  }
  out[0] = out[1] = out[2] = T(0);
  const NodeRows<D> nr(pg, cell, base);
#pragma unroll
  for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
#pragma unroll
    for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
#pragma unroll
      for (int ox = 0; ox < 3; ox++) {
        const int g = nr.at(ox, oy, oz);
        T r[NVP];
        load_rec<NVP>(nodes + (size_t)g * NVP, r);
        const T w = Sw[0][ox] * (D > 1 ? Sw[1][oy] : T(1)) * (D > 2 ? Sw[2][oz] : T(1));
#pragma unroll
        for (int c = 0; c < 3; c++) out[c] += w * r[D + 3 + c];
      }
}

// A_h(u) at the time fraction sig of the field step, A^n + sig (A^{n+1} - A^n)
// (Eq. A-g-s), from the node records (substeps of refinement)
template <int D, typename T>
__device__ __forceinline__ void interp_At(const PGeom &pg, const int cell[3], const T u[3],
                                          const T *__restrict__ nodes, T sig, T out[3],
                                          int order) {
  constexpr int NVP = Rec<D>::NVP;
  int base[3] = {0, 0, 0};
  T Sw[3][3];
#pragma unroll
  for (int l = 0; l < D; l++) {
    base[l] = (int)floor(u[l] + T(0.5));
    spline_val<T>(order, u[l] - T(base[l]), Sw[l]);
  }
  out[0] = out[1] = out[2] = T(0);
  const NodeRows<D> nr(pg, cell, base);
#pragma unroll
  for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
#pragma unroll
    for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
#pragma unroll
      for (int ox = 0; ox < 3; ox++) {
        const int g = nr.at(ox, oy, oz);
        T r[NVP];
        load_rec<NVP>(nodes + (size_t)g * NVP, r);
        const T w = Sw[0][ox] * (D > 1 ? Sw[1][oy] : T(1)) * (D > 2 ? Sw[2][oz] : T(1));
#pragma unroll
        for (int c = 0; c < 3; c++) out[c] += w * (r[D + c] + sig * (r[D + 3 + c] - r[D + c]));
      }
}

// A_h(u) from a component-major FP64 mesh array (step start, energy, deposits)
template <int D, typename T>
__device__ __forceinline__ void point_interp(const PGeom &pg, const int cell[3], const T u[3],
                                             const double *__restrict__ F, T out[3]) {
  int base[3] = {0, 0, 0};
  T Sw[3][3];
#pragma unroll
  for (int l = 0; l < D; l++) {
    base[l] = (int)floor(u[l] + T(0.5));
    spline_val<T>(pg.order, u[l] - T(base[l]), Sw[l]);
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
        const T w = Sw[0][ox] * (D > 1 ? Sw[1][oy] : T(1)) * (D > 2 ? Sw[2][oz] : T(1));
#pragma unroll
        for (int c = 0; c < 3; c++) out[c] += w * (T)__ldg(F + (size_t)c * pg.Ng + g);
      }
}

// A_h(u) from a component-major mesh array in the particle real type
template <int D, typename T>
__device__ __forceinline__ void point_interp_T(const PGeom &pg, const int cell[3], const T u[3],
                                               const T *__restrict__ F, T out[3]) {
  int base[3] = {0, 0, 0};
  T Sw[3][3];
#pragma unroll
  for (int l = 0; l < D; l++) {
    base[l] = (int)floor(u[l] + T(0.5));
    spline_val<T>(pg.order, u[l] - T(base[l]), Sw[l]);
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
        const T w = Sw[0][ox] * (D > 1 ? Sw[1][oy] : T(1)) * (D > 2 ? Sw[2][oz] : T(1));
#pragma unroll
        for (int c = 0; c < 3; c++) out[c] += w * __ldg(F + (size_t)c * pg.Ng + g);
      }
}

// Per-particle constants of the push.
template <typename T>
struct PushConst {
  T q, m, inv_m, mk, inv_mk, hq, a_hc, gamma_n;
  T Pn[3], Am[3], pn[3];
};

// GM-HC canonical step (Eq. gmhc-step) with the HC map of Def. hc-normalized
// generated by B_eff(K), K = D^T - D (Eqs. D-split-skew, beff-KA), and the
// orbit velocity of Eqs. electric-work-velocities, vbar-energy.
// Dm holds D_i A with its columns already in physical units.
template <int D, typename T>
__device__ __forceinline__ void gmhc_push(const PushConst<T> &pc, const T Ap[3], const T gphi[3],
                                          const T Dm[3][3], const T vb[3], T vn[3], T Pn1[3]) {
  T Aep[3], com[3], pm[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    Aep[c] = T(0.5) * (pc.Am[c] + Ap[c]);
    T Dv = T(0);
#pragma unroll
    for (int j = 0; j < D; j++) Dv += Dm[c][j] * vb[j];
    com[c] = pc.hq * (Dv - (c < D ? gphi[c] : T(0)));
    pm[c] = pc.Pn[c] - pc.q * Aep[c] + com[c];
  }
  // B_eff = (K_23, -K_13, K_12) with K_lj = D_jl - D_lj
  auto Dat = [&](int r, int c) -> T { return c < D ? Dm[r][c] : T(0); };
  T tau[3];
  tau[0] = pc.a_hc * (Dat(2, 1) - Dat(1, 2));
  tau[1] = pc.a_hc * (Dat(0, 2) - Dat(2, 0));
  tau[2] = pc.a_hc * (Dat(1, 0) - Dat(0, 1));
  T um[3];
#pragma unroll
  for (int c = 0; c < 3; c++) um[c] = pm[c] * pc.inv_mk;
  const T gm2 = T(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
  const T tau2 = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
  const T sig = gm2 - tau2;
  const T ut = um[0] * tau[0] + um[1] * tau[1] + um[2] * tau[2];
  // gamma_HC^2 = (sig + sqrt(sig^2 + 4 (|tau|^2 + (u.tau)^2))) / 2, Eq. gammaHC
  const T g2 = T(0.5) * (sig + sqrt(sig * sig + T(4) * (tau2 + ut * ut)));
  const T ig = rsqrt(g2);
  T t[3];
#pragma unroll
  for (int c = 0; c < 3; c++) t[c] = tau[c] * ig;
  const T t2 = tau2 * ig * ig;
  const T f = T(2) / (T(1) + t2);
  T us[3], up[3];
  us[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
  us[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
  us[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
  up[0] = um[0] + f * (us[1] * t[2] - us[2] * t[1]);
  up[1] = um[1] + f * (us[2] * t[0] - us[0] * t[2]);
  up[2] = um[2] + f * (us[0] * t[1] - us[1] * t[0]);
  T pp[3], pn1[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    pp[c] = pc.mk * up[c];
    Pn1[c] = pp[c] + pc.q * Aep[c] + com[c];
    pn1[c] = Pn1[c] - pc.q * Ap[c];
  }
  // secant velocities (Eq. Vdg); |p+| = |p-| (Eq. magnetic-kinetic-zero), so
  // gamma(p+) = gamma(p-) = sqrt(1 + |u-|^2)
  const T g_m = sqrt(gm2);
  const T g_n1 =
      sqrt(T(1) + (pn1[0] * pn1[0] + pn1[1] * pn1[1] + pn1[2] * pn1[2]) * pc.inv_mk * pc.inv_mk);
  const T d1 = g_m + pc.gamma_n, d2 = g_n1 + g_m;
  const T rr = T(0.5) * pc.inv_m / (d1 * d2);
  const T cm = rr * d2, cp = rr * d1;
#pragma unroll
  for (int c = 0; c < 3; c++) vn[c] = cm * (pm[c] + pc.pn[c]) + cp * (pn1[c] + pp[c]);
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
  // FP32 contexts: each converged particle's deposit record (two float4 per
  // particle, DepRec), written by the solve pass for the deposit pass; or null
  float4 *drec = nullptr;
};

// sums of NQ values over the CTA, written to out[0 .. NQ)
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
    out[threadIdx.x] = s;
  }
}

// Extra inner sweeps after the value has passed the inner test: none for
// plain types; two for dual numbers, whose tangent converges at the value's
// rate and so is still about as far from its fixed point as the value was.
// The count depends on the value alone, so a dual map evaluation is exactly
// linear in its tangent inputs (the branches of the value decide everything).
template <typename T>
constexpr int kTangentSweeps = 0;
template <>
constexpr int kTangentSweeps<Dual> = 2;

// The gathers of one inner sweep over the straight orbit that starts at
// (cell, off) with velocity vb and lasts tsp of the field step: grad phi^{1/2}
// and D_i A (columns in physical units) averaged along the orbit, and A at
// its end (A^{n+1}, or A(ta + tsp) for a substep).  False when the orbit
// crosses more knot planes than the walk handles.
template <int D, typename T, bool SUB>
__device__ __forceinline__ bool orbit_gather(const int cell[3], const T off[3], const T dtdx[3],
                                             T ta, T tsp, const T *__restrict__ nodes,
                                             const PGeom &pg, const KConst<T> &kc,
                                             const MapScale<T> &ms, const T vb[3], T gphi[3],
                                             T Dm[3][3], T Ap[3], int &npieces, int order) {
  GatherOrbit<D, T, SUB> go;
  go.nodes = nodes;
  go.pg = &pg;
  go.kc = &kc;
  go.pieces = 0;
  go.ta = ta;
  go.tsp = tsp;
  go.order = order;
#pragma unroll
  for (int l = 0; l < 3; l++) {
    go.cell[l] = cell[l];
    go.off[l] = off[l];
    go.del[l] = vb[l] * dtdx[l];
    go.gphi[l] = T(0);
    go.Dm[l][0] = go.Dm[l][1] = go.Dm[l][2] = T(0);
  }
  const bool ok = walk_orbit<D, T>(go.off, go.del, go, order);
  npieces += go.pieces;
  if (!ok) return false;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    gphi[c] = go.gphi[c];
#pragma unroll
    for (int j = 0; j < 3; j++) Dm[c][j] = j < D ? go.Dm[c][j] * ms.inv_dx[j] : go.Dm[c][j];
  }
  T u1[3];
#pragma unroll
  for (int l = 0; l < 3; l++) u1[l] = go.off[l] + go.del[l];
  if (SUB) interp_At<D, T>(pg, cell, u1, nodes, ta + tsp, Ap, order);
  else interp_A1<D, T>(pg, cell, u1, nodes, Ap, order);
  return true;
}

// One particle's inner Picard iteration (Sec. 4.5, reading R6) over the
// straight orbit that starts at (cell, off) and lasts tsp of the field step
// (tsp = 1 unless SUB: then the orbit is the substep [ta, ta + tsp] of a
// refined particle).  vb holds the starting iterate and returns the last one,
// Pn1 the matching P^{n+1}, it the iterations used.  Returns true when the
// inner test passed; otherwise st receives the reason.
template <int D, typename T, bool SUB>
__device__ __forceinline__ bool picard(const PushConst<T> &pc, const int cell[3], const T off[3],
                                       const T dtdx[3], T ta, T tsp, const T *__restrict__ nodes,
                                       const PGeom &pg, const KConst<T> &kc,
                                       const MapScale<T> &ms, T vb[3], T Pn1[3], int &it_out,
                                       int &npieces, unsigned int &st, int order) {
  const T tau_r = kc.tau_r, tau_a = kc.tau_a, kap2 = kc.kappa * kc.kappa;
  unsigned int sl = 0;
  bool conv = false;
  int it, extra = -1;  // sweeps left after the value converged (dual numbers)
#pragma unroll 1
  for (it = 1; it <= kc.inner_max + kTangentSweeps<T>; it++) {
    T gphi[3], Dm[3][3], Ap[3];
    if (!orbit_gather<D, T, SUB>(cell, off, dtdx, ta, tsp, nodes, pg, kc, ms, vb, gphi, Dm, Ap,
                                 npieces, order)) {
      sl |= PIC_ST_PIECES;
      break;
    }
    T vn[3], Pc[3];
    gmhc_push<D, T>(pc, Ap, gphi, Dm, vb, vn, Pc);
    T diff = T(0), nrm = T(0), v2 = T(0);
    bool fin = true;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      fin = fin && isfinite(vn[c]);
      diff = fmax(diff, fabs(vn[c] - vb[c]));
      nrm = fmax(nrm, fabs(vn[c]));
      v2 += vn[c] * vn[c];
    }
    if (!fin) {
      sl |= PIC_ST_NONFINITE;
      break;
    }
    if (v2 >= kap2) {
      sl |= PIC_ST_SUPERLUM;
      break;
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
      vb[c] = vn[c];
      Pn1[c] = Pc[c];
    }
    if constexpr (kTangentSweeps<T> == 0) {
      if (diff <= tau_a + tau_r * nrm) {
        conv = true;
        break;
      }
    } else {
      if (extra < 0 && it <= kc.inner_max && diff <= tau_a + tau_r * nrm)
        extra = kTangentSweeps<T>;
      if (extra == 0) {
        conv = true;
        break;
      }
      if (extra > 0) extra--;
    }
  }
  if (!conv && sl == 0) sl |= PIC_ST_NOCONV;
  st |= sl;
  it_out = it;
  return conv;
}

// The orbit deposit of Eq. orbit-current-energy for one converged (sub)orbit,
// weighted by wgt (the substep's share of the field step; 1 without
// refinement), and on the final pass the particle work and chain-rule sums
// of Sec. 4.4 (pc.Am is A at the orbit's start, dts its duration).
template <int D, typename T, bool FINAL, bool SUB>
__device__ __forceinline__ void deposit_orbit(const PushConst<T> &pc, const int cell[3],
                                              const T off[3], const T dtdx[3], T ta, T tsp, T dts,
                                              T wgt, const T vb[3], const T *__restrict__ nodes,
                                              const T *__restrict__ nodes_u,
                                              double *__restrict__ J, const PGeom &pg,
                                              const KConst<T> &kc, const MapScale<T> &ms, T *win,
                                              const int ref[3], int &npieces, unsigned int &st,
                                              double &work, double &chain, int order) {
  const T qdv = pc.q * ms.inv_dV * wgt;
  DepositOrbit<D, T, FINAL, SUB> dp;
  dp.nodes = nodes;
  dp.nodes_u = nodes_u;
  dp.J = J;
  dp.pg = &pg;
  dp.kc = &kc;
  dp.pieces = 0;
  dp.win = win;
  dp.ta = ta;
  dp.tsp = tsp;
  dp.order = order;
#pragma unroll
  for (int l = 0; l < 3; l++) {
    dp.ref[l] = ref[l];
    dp.cell[l] = cell[l];
    dp.off[l] = off[l];
    dp.del[l] = vb[l] * dtdx[l];
    dp.qv[l] = qdv * vb[l];
    dp.gphi[l] = dp.Ubar[l] = T(0);
    dp.Dm[l][0] = dp.Dm[l][1] = dp.Dm[l][2] = T(0);
  }
  if (!walk_orbit<D, T>(dp.off, dp.del, dp, order)) st |= PIC_ST_PIECES;
  npieces += dp.pieces;
  if (FINAL) {
    T u1[3], Ap[3];
#pragma unroll
    for (int l = 0; l < 3; l++) u1[l] = dp.off[l] + dp.del[l];
    if (SUB) interp_At<D, T>(pg, cell, u1, nodes, ta + tsp, Ap, order);
    else interp_A1<D, T>(pg, cell, u1, nodes, Ap, order);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      T Dv = T(0);
#pragma unroll
      for (int j = 0; j < D; j++) Dv += dp.Dm[c][j] * ms.inv_dx[j] * vb[j];
      T Eb = -(c < D ? dp.gphi[c] : T(0)) - dp.Ubar[c];
      work += (double)(wgt * pc.q * vb[c] * Eb);
      T RA = Ap[c] - pc.Am[c] - dts * (dp.Ubar[c] + Dv);
      chain += (double)RA * (double)RA;
    }
  }
}

constexpr int kMaxSub = 8;  // substeps at the largest refinement depth (3)

// Convergence-triggered particle refinement (Sec. 5.3): the particle's
// full-step solve failed, so it is retried with 2, 4, .. 2^refine_max equal
// substeps of the field step (the field step itself is unchanged).  Substep
// [ta, ta + tsp] starts where the previous one ended, with A^- = A(ta) at its
// start and the cold start v(p) (reading R5), and sees the time-linear
// potential of Eq. A-g-s and the step's grad phi^{1/2}.  When every substep
// of a level converges, each deposits its orbit current weighted by tsp (the
// orbit-averaged current); vbar returns the mean substep orbit velocity (so
// that x^n + dt vbar is the end point) and Pnew the last substep's P.
template <int D, typename T, bool FINAL>
__device__ __noinline__ bool refine_particle(const PushConst<T> &pc0, const int cell0[3],
                                             const T off0[3], const T *__restrict__ nodes,
                                             const T *__restrict__ nodes_u,
                                             double *__restrict__ J, const PGeom &pg,
                                             const KConst<T> &kc, const MapScale<T> &ms, T *win,
                                             const int ref[3], T vbar[3], T Pnew[3], int &iters,
                                             int &npieces, unsigned int &st, double &work,
                                             double &chain) {
  const int levels = kc.refine_max < 3 ? kc.refine_max : 3;
  for (int lvl = 1; lvl <= levels; lvl++) {
    const int nsub = 1 << lvl;
    const T tsp = T(1) / T(nsub), dts = kc.dt * tsp;
    T dtdx[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int l = 0; l < D; l++) dtdx[l] = dts * ms.inv_dx[l];
    int cs[kMaxSub][3];
    T os[kMaxSub][3], vs[kMaxSub][3], As[kMaxSub][3];
    int cell[3] = {cell0[0], cell0[1], cell0[2]};
    T off[3] = {off0[0], off0[1], off0[2]};
    T P[3] = {pc0.Pn[0], pc0.Pn[1], pc0.Pn[2]};
    int its = 0;
    bool ok = true;
    for (int sub = 0; sub < nsub; sub++) {
      const T ta = T(sub) * tsp;
      PushConst<T> pc = pc0;
      pc.hq = T(0.5) * pc.q * dts;
      pc.a_hc = pc.hq * pc.inv_m;
      interp_At<D, T>(pg, cell, off, nodes, ta, pc.Am, kc.order);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        pc.Pn[c] = P[c];
        pc.pn[c] = P[c] - pc.q * pc.Am[c];
      }
      pc.gamma_n = sqrt(T(1) + (pc.pn[0] * pc.pn[0] + pc.pn[1] * pc.pn[1] +
                                pc.pn[2] * pc.pn[2]) * pc.inv_mk * pc.inv_mk);
      const T ig = T(1) / (pc.m * pc.gamma_n);
      T vb[3], Pn1[3];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        vb[c] = pc.pn[c] * ig;
        Pn1[c] = P[c];
      }
      int it = 0;
      unsigned int sl = 0;
      if (!picard<D, T, true>(pc, cell, off, dtdx, ta, tsp, nodes, pg, kc, ms, vb, Pn1, it,
                              npieces, sl, kc.order)) {
        ok = false;
        break;
      }
      its += it;
#pragma unroll
      for (int l = 0; l < 3; l++) {
        cs[sub][l] = cell[l];
        os[sub][l] = off[l];
        vs[sub][l] = vb[l];
        As[sub][l] = pc.Am[l];
      }
#pragma unroll
      for (int l = 0; l < D; l++) {  // to the substep's end point
        const T u = off[l] + dtdx[l] * vb[l];
        const T shf = floor(u + T(0.5));
        cell[l] = (cell[l] + (int)shf) & pg.mask[l];
        off[l] = u - shf;
      }
#pragma unroll
      for (int c = 0; c < 3; c++) P[c] = Pn1[c];
    }
    if (!ok) continue;
    for (int sub = 0; sub < nsub; sub++) {
      PushConst<T> pc = pc0;
#pragma unroll
      for (int c = 0; c < 3; c++) pc.Am[c] = As[sub][c];
      deposit_orbit<D, T, FINAL, true>(pc, cs[sub], os[sub], dtdx, T(sub) * tsp, tsp, dts, tsp,
                                       vs[sub], nodes, nodes_u, J, pg, kc, ms, win, ref, npieces,
                                       st, work, chain, kc.order);
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
      T v = T(0);
      for (int sub = 0; sub < nsub; sub++) v += vs[sub][c];
      vbar[c] = v * tsp;
      Pnew[c] = P[c];
    }
    iters = its;
    return true;
  }
  return false;
}

// The particle map of one thread (particle i) of a CTA of kPT threads: inner
// Picard iteration, deposit, counters.  pv.np bounds the particles of this
// CTA's problem (threads with i >= pv.np only join the warp and block
// collectives), pg / nodes / nodes_u / J / kc / ms / cnt describe that
// problem, and psum[0..2) receives the CTA's final-pass partial sums.
// GEN = false is the common path, compiled for quadratic shapes without
// refinement; GEN = true reads the shape degree from kc and compiles in the
// refinement retry (kc.refine_max > 0).  Keeping both out of the common
// path leaves it with no call and no per-point branch on the degree.
template <int D, typename T, bool FINAL, bool GEN = false, typename S = T>
__device__ __forceinline__ void map_block(const PView<S> &pv, const int64_t i_slot,
                                          const T *__restrict__ nodes,
                                          const T *__restrict__ nodes_u, double *__restrict__ J,
                                          const PGeom &pg, const KConst<T> &kc,
                                          const MapScale<T> &ms,
                                          EvalCounters *__restrict__ cnt,
                                          double *__restrict__ psum) {
  // Piece-count grouping: a warp walks as many orbit pieces as its slowest
  // lane, and most orbits have one piece while a few cross one or two knot
  // planes.  So the CTA's particles are reordered (stably) by the number of
  // half-integer planes their start velocity would cross, predicted from
  // the offset and v(p^n), and thread t takes the t-th of that order: the
  // orbits that cross gather in few warps.  The order changes only which
  // thread computes which particle.
  __shared__ int s_perm[kPT];
  __shared__ int s_wcnt[kPT / 32][4];
  {
    int cls = 3;  // empty slots go last
    if (i_slot < pv.np) {
      cls = 0;
#pragma unroll
      for (int l = 0; l < D; l++) {
        const T u = (T)pv.off[l * pv.cap + i_slot] +
                    (T)(kc.warm ? pv.vbar[l * pv.cap + i_slot] : pv.v0[l * pv.cap + i_slot]) *
                        kc.dt * ms.inv_dx[l];
        cls += (u >= T(0.5) || u < T(-0.5)) ? 1 : 0;
      }
      cls = cls < 2 ? cls : 2;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned mine = 0;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const unsigned b = __ballot_sync(0xffffffffu, cls == c);
      if (lane == 0) s_wcnt[wid][c] = __popc(b);
      if (cls == c) mine = b;
    }
    __syncthreads();
    int pos = __popc(mine & ((1u << lane) - 1u));
    for (int c = 0; c < cls; c++)
      for (int w = 0; w < kPT / 32; w++) pos += s_wcnt[w][c];
    for (int w = 0; w < wid; w++) pos += s_wcnt[w][cls];
    s_perm[pos] = threadIdx.x;
    __syncthreads();
  }
  const int64_t i = i_slot - threadIdx.x + s_perm[threadIdx.x];
  const bool active = i < pv.np;
  double work = 0.0, chain = 0.0;
  int iters = 0, npieces = 0, refined = 0;
  unsigned int st = 0;
  // FP32 deposit window of this warp (see WarpWin): reference cell = the
  // cell of lane 0's particle, columns zeroed by their lanes
  constexpr bool kWin = WarpWin<D>::kOn && sizeof(T) == 4;
  __shared__ T s_win[kWin ? (kPT / 32) * WarpWin<D>::NE * 32 : 1];
  T *win_warp = s_win + (size_t)(threadIdx.x >> 5) * WarpWin<D>::NE * 32;
  T *win_col = kWin ? win_warp + (threadIdx.x & 31) : nullptr;
  int ref[3] = {0, 0, 0};
  if constexpr (kWin) {
    const int64_t i0 = __shfl_sync(0xffffffffu, i, 0);  // lane 0's particle
    if (i0 < pv.np) {
#pragma unroll
      for (int l = 0; l < D; l++) ref[l] = pv.cell[l * pv.cap + i0];
    }
    for (int e = 0; e < WarpWin<D>::NE; e++) win_col[e * 32] = T(0);
  }
  if (active) {
    const int64_t cap = pv.cap;
    const int s_id = pv.sp[i];
    PushConst<T> pc;
    pc.q = (T)(pv.w[i] * kc.qs[s_id]);
    pc.m = (T)(pv.w[i] * kc.ms[s_id]);
    const T kap = kc.kappa, dt = kc.dt;
    pc.inv_m = T(1) / pc.m;
    pc.mk = pc.m * kap;
    pc.inv_mk = pc.inv_m / kap;
    pc.hq = T(0.5) * pc.q * dt;
    pc.a_hc = pc.hq * pc.inv_m;
    int cell[3] = {0, 0, 0};
    T off[3] = {T(0), T(0), T(0)};
    T dtdx[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int l = 0; l < D; l++) {
      cell[l] = pv.cell[l * cap + i];
      off[l] = (T)pv.off[l * cap + i];
      dtdx[l] = dt * ms.inv_dx[l];
    }
    T vb[3], Pn1[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      pc.Pn[c] = (T)pv.P[c * cap + i];
      pc.Am[c] = (T)pv.Am[c * cap + i];
      pc.pn[c] = pc.Pn[c] - pc.q * pc.Am[c];
      vb[c] = (T)(kc.warm ? pv.vbar[c * cap + i] : pv.v0[c * cap + i]);
      Pn1[c] = pc.Pn[c];
    }
    pc.gamma_n = sqrt(T(1) + (pc.pn[0] * pc.pn[0] + pc.pn[1] * pc.pn[1] + pc.pn[2] * pc.pn[2]) *
                                 pc.inv_mk * pc.inv_mk);
    const int order = GEN ? kc.order : 2;
    int it = 0;
    unsigned int st0 = 0;
    bool conv = picard<D, T, false>(pc, cell, off, dtdx, T(0), T(1), nodes, pg, kc, ms, vb, Pn1,
                                    it, npieces, st0, order);
    iters = conv ? it : -1;
    if (conv) {
      deposit_orbit<D, T, FINAL, false>(pc, cell, off, dtdx, T(0), T(1), dt, T(1), vb, nodes,
                                        nodes_u, J, pg, kc, ms, win_col, ref, npieces, st, work,
                                        chain, order);
    } else if (GEN && kc.refine_max > 0) {
      T vr[3], Pr[3];
      int itr = 0;
      if (refine_particle<D, T, FINAL>(pc, cell, off, nodes, nodes_u, J, pg, kc, ms, win_col, ref,
                                       vr, Pr, itr, npieces, st, work, chain)) {
        conv = true;
        refined = 1;
        iters = itr;
        st0 = 0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          vb[c] = vr[c];
          Pn1[c] = Pr[c];
        }
      }
    }
    st |= st0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      pv.vbar[c * cap + i] = (S)vb[c];
      pv.Pnew[c * cap + i] = (S)Pn1[c];
    }
    pv.iters[i] = iters;
  }
  if constexpr (kWin) {
    // reduce the 32 columns of the warp window (rotated so that the lanes read
    // 32 different banks) and flush each touched entry with one FP64 atomic
    __syncwarp();
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < WarpWin<D>::NE; e += 32) {
      const T *rowp = win_warp + (size_t)e * 32;
      T sum = T(0);
#pragma unroll 8
      for (int l = 0; l < 32; l++) sum += rowp[(l + lane) & 31];
      if (sum != T(0)) {
        const int node = e / 3, c = e - 3 * node;
        const int rx = node % WarpWin<D>::N0 + WarpWin<D>::LO0;
        const int ry = node / WarpWin<D>::N0 + WarpWin<D>::LO1;
        int g = (ref[0] + rx) & pg.mask[0];
        if (D > 1) g += pg.n0 * ((ref[1] + ry) & pg.mask[1]);
        atomicAdd(J + (size_t)c * pg.Ng + g, widen(sum));
      }
    }
  }
  // counters: integer warp reductions, one atomic per warp
  if (st) atomicOr(&cnt->status, st);
  const unsigned it_sum = __reduce_add_sync(0xffffffffu, (unsigned)(iters > 0 ? iters : 0));
  const unsigned pc_sum = __reduce_add_sync(0xffffffffu, (unsigned)npieces);
  const unsigned rf_sum = __reduce_add_sync(0xffffffffu, (unsigned)refined);
  const int mx = __reduce_max_sync(0xffffffffu, iters);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&cnt->inner_sum, (unsigned long long)it_sum);
    atomicAdd(&cnt->pieces, (unsigned long long)pc_sum);
    if (rf_sum) atomicAdd(&cnt->refined, (unsigned long long)rf_sum);
    if (mx > 0) atomicMax(&cnt->inner_max, mx);
  }
  if (FINAL) {
    double v[2] = {work, chain};
    block_sums<2>(v, psum);
  }
}

// the global nanosecond timer
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---- the particle map with lane refill -----------------------------------
//
// A warp executes each inner sweep for as long as its slowest lane still
// iterates, so in map_block the lanes whose particles converged early idle
// until the warp's last particle converges.  map_chunk_solve removes that
// wait: a CTA owns a chunk of kRefillOf<T> * kPT particles, and a lane whose
// particle has converged (or failed) stores it and takes the next particle of
// the chunk from a shared counter, so the sweeps run with full warps until
// the chunk runs dry.  The chunk is ordered by the predicted number of knot
// planes crossed (as in map_block) so that the particles a warp holds at one
// time walk similar numbers of orbit pieces.  The deposits follow from the
// stored orbit velocities (map_chunk_deposit): in a second launch for FP32
// arithmetic (k_map_solve, k_map_deposit), in the same CTA after a barrier
// for FP64 (k_map_fused).  Every particle's arithmetic is that of map_block:
// only which lane computes it, and when, changes.
// Chunk of particles per CTA: 8 x kPT for FP64 arithmetic (longer chunks
// shorten the share of the drain at each chunk's end), 4 x kPT for FP32
// (whose inputs are staged in shared memory, chunk by chunk).
template <typename T>
constexpr int kRefillOf = sizeof(T) == 8 ? 8 : 4;
template <typename T>
constexpr int kChunkOf = kRefillOf<T> * kPT;
constexpr int kChunk = kChunkOf<float>;        // the FP32 staging chunk
constexpr int kChunkMax = kChunkOf<double>;    // the longest chunk
static_assert(kChunkMax % kChunk == 0, "the staging chunk divides the capacity granule");

// one particle's inner solve between sweeps
template <int D, typename T>
struct LaneSolve {
  PushConst<T> pc;
  int cell[3];
  T off[3], dtdx[3], vb[3], Pn1[3];
  int it;
};

// Where a particle's step inputs are read: the particle arrays in global
// memory (GSrc, index = particle slot), or one chunk of them staged in
// shared memory (StSrc, index = position in the chunk).  vel is v^0, or the
// last orbit velocity when the inner iteration is warm-started.
template <typename S>
struct GSrc {
  const PView<S> *pv;
  const S *vel;
  __device__ __forceinline__ int cell(int l, int64_t i) const { return pv->cell[l * pv->cap + i]; }
  __device__ __forceinline__ S off(int l, int64_t i) const { return pv->off[l * pv->cap + i]; }
  __device__ __forceinline__ S P(int c, int64_t i) const { return pv->P[c * pv->cap + i]; }
  __device__ __forceinline__ S Am(int c, int64_t i) const { return pv->Am[c * pv->cap + i]; }
  __device__ __forceinline__ S v(int c, int64_t i) const { return vel[c * pv->cap + i]; }
  __device__ __forceinline__ double w(int64_t i) const { return pv->w[i]; }
  __device__ __forceinline__ int sp(int64_t i) const { return pv->sp[i]; }
};

// One chunk of particle inputs in shared memory, one array per component of
// kChunk entries: cell (D), offset (D), P (3), A^- (3), start velocity (3),
// weight, species.  Every array starts on a 16-byte boundary (kChunk * 4 is).
template <int D, typename S>
struct Stage {
  static constexpr int kCell = 0;
  static constexpr int kOff = kCell + D * kChunk * 4;
  static constexpr int kP = kOff + D * kChunk * (int)sizeof(S);
  static constexpr int kAm = kP + 3 * kChunk * (int)sizeof(S);
  static constexpr int kV = kAm + 3 * kChunk * (int)sizeof(S);
  static constexpr int kW = kV + 3 * kChunk * (int)sizeof(S);
  static constexpr int kSp = kW + kChunk * 8;
  static constexpr int kBytes = kSp + kChunk * 4;
};

template <int D, typename S>
struct StSrc {
  const char *base;
  __device__ __forceinline__ int cell(int l, int64_t k) const {
    return reinterpret_cast<const int *>(base + Stage<D, S>::kCell)[l * kChunk + k];
  }
  __device__ __forceinline__ S off(int l, int64_t k) const {
    return reinterpret_cast<const S *>(base + Stage<D, S>::kOff)[l * kChunk + k];
  }
  __device__ __forceinline__ S P(int c, int64_t k) const {
    return reinterpret_cast<const S *>(base + Stage<D, S>::kP)[c * kChunk + k];
  }
  __device__ __forceinline__ S Am(int c, int64_t k) const {
    return reinterpret_cast<const S *>(base + Stage<D, S>::kAm)[c * kChunk + k];
  }
  __device__ __forceinline__ S v(int c, int64_t k) const {
    return reinterpret_cast<const S *>(base + Stage<D, S>::kV)[c * kChunk + k];
  }
  __device__ __forceinline__ double w(int64_t k) const {
    return reinterpret_cast<const double *>(base + Stage<D, S>::kW)[k];
  }
  __device__ __forceinline__ int sp(int64_t k) const {
    return reinterpret_cast<const int *>(base + Stage<D, S>::kSp)[k];
  }
};

template <int D, typename T, typename Src>
__device__ __forceinline__ void lane_init_from(LaneSolve<D, T> &ls, const Src &src, int64_t i,
                                               const KConst<T> &kc, const MapScale<T> &ms) {
  const int s_id = src.sp(i);
  PushConst<T> &pc = ls.pc;
  if constexpr (std::is_same<T, float>::value) {
    // FP32: the weight rounded once, then FP32 products (no FP64 arithmetic,
    // whose pipe is 1/64 of the FP32 one)
    const float wf = (float)src.w(i);
    pc.q = wf * kc.qT[s_id];
    pc.m = wf * kc.mT[s_id];
  } else {
    pc.q = (T)(src.w(i) * kc.qs[s_id]);
    pc.m = (T)(src.w(i) * kc.ms[s_id]);
  }
  const T kap = kc.kappa, dt = kc.dt;
  pc.inv_m = T(1) / pc.m;
  pc.mk = pc.m * kap;
  pc.inv_mk = pc.inv_m / kap;
  pc.hq = T(0.5) * pc.q * dt;
  pc.a_hc = pc.hq * pc.inv_m;
#pragma unroll
  for (int l = 0; l < 3; l++) {
    ls.cell[l] = l < D ? src.cell(l, i) : 0;
    ls.off[l] = l < D ? (T)src.off(l, i) : T(0);
    ls.dtdx[l] = l < D ? dt * ms.inv_dx[l] : T(0);
  }
#pragma unroll
  for (int c = 0; c < 3; c++) {
    pc.Pn[c] = (T)src.P(c, i);
    pc.Am[c] = (T)src.Am(c, i);
    pc.pn[c] = pc.Pn[c] - pc.q * pc.Am[c];
    ls.vb[c] = (T)src.v(c, i);
    ls.Pn1[c] = pc.Pn[c];
  }
  pc.gamma_n = sqrt(T(1) + (pc.pn[0] * pc.pn[0] + pc.pn[1] * pc.pn[1] + pc.pn[2] * pc.pn[2]) *
                               pc.inv_mk * pc.inv_mk);
  ls.it = 0;
}

template <int D, typename T, typename S>
__device__ __forceinline__ void lane_init(LaneSolve<D, T> &ls, const PView<S> &pv, int64_t i,
                                          const KConst<T> &kc, const MapScale<T> &ms) {
  const GSrc<S> src{&pv, kc.warm ? pv.vbar : pv.v0};
  lane_init_from<D, T>(ls, src, i, kc, ms);
}

// One inner sweep of the particle a lane holds (the body of picard's loop):
// 0 = not converged yet, 1 = converged, 2 = failed (status bits in sl).
template <int D, typename T>
__device__ __forceinline__ int lane_sweep(LaneSolve<D, T> &ls, const T *__restrict__ nodes,
                                          const PGeom &pg, const KConst<T> &kc,
                                          const MapScale<T> &ms, int &npieces,
                                          unsigned int &sl) {
  ls.it++;
  T gphi[3], Dm[3][3], Ap[3];
  if (!orbit_gather<D, T, false>(ls.cell, ls.off, ls.dtdx, T(0), T(1), nodes, pg, kc, ms, ls.vb,
                                 gphi, Dm, Ap, npieces, 2)) {
    sl |= PIC_ST_PIECES;
    return 2;
  }
  T vn[3], Pc[3];
  gmhc_push<D, T>(ls.pc, Ap, gphi, Dm, ls.vb, vn, Pc);
  T diff = T(0), nrm = T(0), v2 = T(0);
  bool fin = true;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    fin = fin && isfinite(vn[c]);
    diff = fmax(diff, fabs(vn[c] - ls.vb[c]));
    nrm = fmax(nrm, fabs(vn[c]));
    v2 += vn[c] * vn[c];
  }
  if (!fin) {
    sl |= PIC_ST_NONFINITE;
    return 2;
  }
  if (v2 >= kc.kappa * kc.kappa) {
    sl |= PIC_ST_SUPERLUM;
    return 2;
  }
#pragma unroll
  for (int c = 0; c < 3; c++) {
    ls.vb[c] = vn[c];
    ls.Pn1[c] = Pc[c];
  }
  if (diff <= kc.tau_a + kc.tau_r * nrm) return 1;
  if (ls.it >= kc.inner_max) {
    sl |= PIC_ST_NOCONV;
    return 2;
  }
  return 0;
}

// Orders the nvalid particles of the chunk at c0 (in src's indexing) by the
// number of knot planes (0, 1, 2 or more) that a straight orbit with velocity
// src.v crosses (stable, deterministic), into s_order.  Ends with a barrier.
template <int D, typename T, typename Src>
__device__ __forceinline__ void order_chunk(const Src &src, const int64_t c0, int nvalid,
                                            const KConst<T> &kc, const MapScale<T> &ms,
                                            int *s_order) {
  __shared__ int s_wcnt[kRefillOf<T>][kPT / 32][4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int cls_of[kRefillOf<T>];
  unsigned mine[kRefillOf<T>];
#pragma unroll
  for (int q = 0; q < kRefillOf<T>; q++) {
    const int k = q * kPT + threadIdx.x;
    int cls = 3;
    if (k < nvalid) {
      const int64_t i = c0 + k;
      cls = 0;
#pragma unroll
      for (int l = 0; l < D; l++) {
        const T u = (T)src.off(l, i) + (T)src.v(l, i) * kc.dt * ms.inv_dx[l];
        cls += (u >= T(0.5) || u < T(-0.5)) ? 1 : 0;
      }
      cls = cls < 2 ? cls : 2;
    }
    cls_of[q] = cls;
    mine[q] = 0;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const unsigned b = __ballot_sync(0xffffffffu, cls == c);
      if (lane == 0) s_wcnt[q][wid][c] = __popc(b);
      if (cls == c) mine[q] = b;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kRefillOf<T>; q++) {
    const int cls = cls_of[q];
    int pos = __popc(mine[q] & ((1u << lane) - 1u));
    for (int c = 0; c < cls; c++)
      for (int qq = 0; qq < kRefillOf<T>; qq++)
        for (int w = 0; w < kPT / 32; w++) pos += s_wcnt[qq][w][c];
    for (int qq = 0; qq < q; qq++)
      for (int w = 0; w < kPT / 32; w++) pos += s_wcnt[qq][w][cls];
    for (int w = 0; w < wid; w++) pos += s_wcnt[q][w][cls];
    s_order[pos] = q * kPT + threadIdx.x;
  }
  __syncthreads();
}

// Bulk asynchronous copies (cp.async.bulk) from global into shared memory,
// completed on an mbarrier, and a wait on it with a time limit.
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// bytes: a multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned phase) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return done != 0;
}
// true when the phase completed; false after limit_ns (or 2^24 polls)
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned phase,
                                          unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0; it < (1u << 24); it++) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((it & 31u) == 31u && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

constexpr unsigned long long kStageWaitNs = 200000000ull;  // 0.2 s: copies take microseconds

// Stages the inputs of the chunk of `chunk` particle slots at c0 (a multiple
// of kPT, at most kChunk; the capacity is a whole number of the longest
// chunks, so every copy stays inside its array and starts on a 16-byte
// boundary) into st by one thread's bulk copies; every thread then waits.
// False (and PIC_ST_WAIT set) if the copies did not complete in time.
template <int D, typename S>
__device__ __forceinline__ bool stage_chunk(const PView<S> &pv, const S *__restrict__ vel,
                                            int64_t c0, int chunk, char *st,
                                            unsigned long long *bar,
                                            EvalCounters *__restrict__ cnt) {
  using L = Stage<D, S>;
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned bs = chunk * (unsigned)sizeof(S), b4 = chunk * 4u;
    mbar_expect_tx(bar, D * b4 + (D + 9) * bs + chunk * 8u + b4);
    const int64_t cap = pv.cap;
#pragma unroll
    for (int l = 0; l < D; l++) {
      bulk_g2s(st + L::kCell + l * kChunk * 4, pv.cell + l * cap + c0, b4, bar);
      bulk_g2s(st + L::kOff + l * kChunk * sizeof(S), pv.off + l * cap + c0, bs, bar);
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
      bulk_g2s(st + L::kP + c * kChunk * sizeof(S), pv.P + c * cap + c0, bs, bar);
      bulk_g2s(st + L::kAm + c * kChunk * sizeof(S), pv.Am + c * cap + c0, bs, bar);
      bulk_g2s(st + L::kV + c * kChunk * sizeof(S), vel + c * cap + c0, bs, bar);
    }
    bulk_g2s(st + L::kW, pv.w + c0, chunk * 8u, bar);
    bulk_g2s(st + L::kSp, pv.sp + c0, b4, bar);
  }
  const bool ok = mbar_wait(bar, 0, kStageWaitNs);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicOr(&cnt->status, PIC_ST_WAIT);
    mbar_wait(bar, 0, kStageWaitNs);  // let copies in flight land before the CTA exits
    return false;
  }
  return true;
}

// The deposit record of one particle, written by the FP32 solve pass when the
// particle's inner solve ends and read by the deposit pass as two coalesced
// 16-byte loads: [cell x | cell y << 16 (int bits), offset x, offset y,
// crossing class (int bits: 0, 1, 2 knot planes or more; 3 = failed)] and
// [orbit velocity (3), charge q].
template <int D>
__device__ __forceinline__ void drec_write(float4 *rec, const LaneSolve<D, float> &ls, int cls) {
  const int cpk = ls.cell[0] | (D > 1 ? (ls.cell[1] << 16) : 0);
  rec[0] = make_float4(__int_as_float(cpk), ls.off[0], D > 1 ? ls.off[1] : 0.0f,
                       __int_as_float(cls));
  rec[1] = make_float4(ls.vb[0], ls.vb[1], ls.vb[2], ls.pc.q);
}

// the number of knot planes (capped at 2) the orbit from off with velocity vb crosses
template <int D, typename T>
__device__ __forceinline__ int crossing_class(const T off[3], const T vb[3], const T dtdx[3]) {
  int cls = 0;
#pragma unroll
  for (int l = 0; l < D; l++) {
    const T u = off[l] + vb[l] * dtdx[l];
    cls += (u >= T(0.5) || u < T(-0.5)) ? 1 : 0;
  }
  return cls < 2 ? cls : 2;
}

// The inner solves of the particle map over one chunk of nr * kPT particle
// slots (nr <= kRefillOf<T>) starting at c0 (the common path: quadratic
// shapes, no refinement):
// every particle's orbit velocity, P^{n+1} and inner count (-1 on failure)
// are stored for the deposit pass (map_chunk_deposit).  With a stage buffer
// (stg, bar non-null: FP32 arithmetic on FP32 storage) the chunk's inputs are
// first copied to shared memory, and the ordering and every refill read them
// there.
template <int D, typename T, typename S>
__device__ __forceinline__ void map_chunk_solve(const PView<S> &pv, const int64_t c0,
                                                const T *__restrict__ nodes, const PGeom &pg,
                                                const KConst<T> &kc, const MapScale<T> &ms,
                                                EvalCounters *__restrict__ cnt, int *s_order,
                                                char *stg, unsigned long long *bar, int nr) {
  __shared__ int s_next;
  const int lane = threadIdx.x & 31;
  const int chunk = nr * kPT;
  const int64_t nvalid64 = pv.np - c0;
  const int nvalid = nvalid64 < chunk ? (int)nvalid64 : chunk;
  if (threadIdx.x == 0) s_next = 0;
  const S *vel = kc.warm ? pv.vbar : pv.v0;
  // a chunk that would reach past the arrays (never, with the host's choice
  // of chunk length) reads them in place instead
  if (stg && c0 + chunk > pv.cap) stg = nullptr;
  if (stg) {
    if (!stage_chunk<D, S>(pv, vel, c0, chunk, stg, bar, cnt)) return;
    // 1. order the chunk by predicted crossing class
    order_chunk<D, T>(StSrc<D, S>{stg}, 0, nvalid, kc, ms, s_order);
  } else {
    order_chunk<D, T>(GSrc<S>{&pv, vel}, c0, nvalid, kc, ms, s_order);
  }
  // 2. the inner solves, lanes refilled from the chunk
  int npieces = 0, mx_it = 0;
  unsigned it_sum = 0;
  unsigned int st = 0;
  LaneSolve<D, T> ls;
  int k = atomicAdd(&s_next, 1);
  bool have = k < nvalid;
  int kk = have ? s_order[k] : 0;
  int64_t i = c0 + kk;
  const StSrc<D, S> ssrc{stg};
  const GSrc<S> gsrc{&pv, vel};
  if (have) {
    if (stg) lane_init_from<D, T>(ls, ssrc, kk, kc, ms);
    else lane_init_from<D, T>(ls, gsrc, i, kc, ms);
  }
  while (__any_sync(0xffffffffu, have)) {
    if (have) {
      unsigned int sl = 0;
      const int r = lane_sweep<D, T>(ls, nodes, pg, kc, ms, npieces, sl);
      if (r != 0) {
        const int64_t cap = pv.cap;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          pv.vbar[c * cap + i] = (S)ls.vb[c];
          pv.Pnew[c * cap + i] = (S)ls.Pn1[c];
        }
        pv.iters[i] = r == 1 ? ls.it : -1;
        if constexpr (std::is_same<T, float>::value && std::is_same<S, float>::value && D < 3) {
          if (pv.drec)
            drec_write<D>(pv.drec + 2 * i, ls, r == 1 ? crossing_class<D, T>(ls.off, ls.vb, ls.dtdx) : 3);
        }
        if (r == 1) {
          it_sum += (unsigned)ls.it;
          mx_it = ls.it > mx_it ? ls.it : mx_it;
        } else {
          st |= sl;
        }
        k = atomicAdd(&s_next, 1);
        have = k < nvalid;
        if (have) {
          kk = s_order[k];
          i = c0 + kk;
          if (stg) lane_init_from<D, T>(ls, ssrc, kk, kc, ms);
          else lane_init_from<D, T>(ls, gsrc, i, kc, ms);
        }
      }
    }
  }
  // counters: integer warp reductions, one atomic per warp
  if (st) atomicOr(&cnt->status, st);
  const unsigned it_w = __reduce_add_sync(0xffffffffu, it_sum);
  const unsigned pc_w = __reduce_add_sync(0xffffffffu, (unsigned)npieces);
  const int mx = __reduce_max_sync(0xffffffffu, mx_it);
  if (lane == 0) {
    atomicAdd(&cnt->inner_sum, (unsigned long long)it_w);
    atomicAdd(&cnt->pieces, (unsigned long long)pc_w);
    if (mx > 0) atomicMax(&cnt->inner_max, mx);
  }
}

// What the deposit of one particle reads: position, orbit velocity, charge.
template <typename T>
struct DepIn {
  int cell[3];
  T off[3], vb[3];
  T q;
};

// the deposit inputs held by one deposit record (drec_write)
template <int D, typename T>
__device__ __forceinline__ void dep_from_rec(DepIn<T> &o, const float4 a, const float4 b) {
  const int cpk = __float_as_int(a.x);
  o.cell[0] = D > 1 ? (cpk & 0xffff) : cpk;
  o.cell[1] = D > 1 ? (cpk >> 16) : 0;
  o.cell[2] = 0;
  o.off[0] = (T)a.y;
  o.off[1] = (T)a.z;
  o.off[2] = T(0);
  o.vb[0] = (T)b.x;
  o.vb[1] = (T)b.y;
  o.vb[2] = (T)b.z;
  o.q = (T)b.w;
}

// from the particle arrays, or (rec non-null) from the particle's deposit
// record (drec_write)
template <int D, typename T, typename S>
__device__ __forceinline__ void dep_load(DepIn<T> &o, const PView<S> &pv, int64_t i,
                                         const KConst<T> &kc, const float4 *rec) {
  if (rec) {
    dep_from_rec<D, T>(o, rec[2 * i], rec[2 * i + 1]);
    return;
  }
#pragma unroll
  for (int l = 0; l < 3; l++) {
    o.cell[l] = l < D ? pv.cell[l * pv.cap + i] : 0;
    o.off[l] = l < D ? (T)pv.off[l * pv.cap + i] : T(0);
    o.vb[l] = (T)pv.vbar[l * pv.cap + i];
  }
  const int s_id = pv.sp[i];
  if constexpr (std::is_same<T, float>::value) o.q = (float)pv.w[i] * kc.qT[s_id];
  else o.q = (T)(pv.w[i] * kc.qs[s_id]);
}

// The orbit deposits of one chunk from the stored orbit velocities (Eq.
// orbit-current-energy), and on the final pass the particle sides of the
// work and chain-rule sums (added to the thread's work and chain).  Lanes take the
// particles in order of the knot planes their orbits cross, so that a warp's
// lanes walk similar numbers of pieces.  FP32 in 1D and 2D: warp w deposits
// the chunk slots [w R, (w + 1) R), R = kRefillOf<T> * 32, ordered within that
// range; the particles are sorted by cell, so the range lies in one or two
// neighbouring cells, and one warp window, referenced to the range's first
// cell, collects all kRefillOf<T> rounds (cleared and summed once per chunk).
// FP64 and 3D: the whole chunk is ordered and deposited with global atomics.
template <int D, typename T, bool FINAL, typename S>
__device__ __forceinline__ void map_chunk_deposit(const PView<S> &pv, const int64_t c0,
                                                  const T *__restrict__ nodes,
                                                  const T *__restrict__ nodes_u,
                                                  double *__restrict__ J, const PGeom &pg,
                                                  const KConst<T> &kc, const MapScale<T> &ms,
                                                  EvalCounters *__restrict__ cnt,
                                                  double &work, double &chain, int *s_order,
                                                  int nr) {
  constexpr int R = kRefillOf<T> * 32;  // the longest warp range
  constexpr bool kWin = WarpWin<D>::kOn && sizeof(T) == 4;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int chunk = nr * kPT;
  const int64_t nvalid64 = pv.np - c0;
  const int nvalid = nvalid64 < chunk ? (int)nvalid64 : chunk;
  int npieces = 0;
  unsigned int st = 0;
  if constexpr (kWin) {
    __shared__ T s_win[(kPT / 32) * WarpWin<D>::NE * 32];
    __shared__ short s_dord[kPT / 32][R];
    const int r0 = wid * nr * 32;  // this warp's range: nr rounds of 32
    // plain passes read the deposit records the solve pass wrote, if any
    const float4 *rec = FINAL ? nullptr : pv.drec;
    int cls_q[kRefillOf<T>];
#pragma unroll
    for (int q = 0; q < kRefillOf<T>; q++) {
      const int k = r0 + q * 32 + lane;
      int cls = 3;  // empty slot, failed particle, or a round past nr: last
      if (rec) {
        if (q < nr && k < nvalid) cls = __float_as_int(rec[2 * (c0 + k)].w);
      } else if (q < nr && k < nvalid && pv.iters[c0 + k] > 0) {
        const int64_t i = c0 + k;
        cls = 0;
#pragma unroll
        for (int l = 0; l < D; l++) {
          const T u = (T)pv.off[l * pv.cap + i] + (T)pv.vbar[l * pv.cap + i] * kc.dt * ms.inv_dx[l];
          cls += (u >= T(0.5) || u < T(-0.5)) ? 1 : 0;
        }
        cls = cls < 2 ? cls : 2;
      }
      cls_q[q] = cls;
    }
    // stable order by class (class, then round, then lane): the start of
    // round q's slots of class c is warp-uniform, from the ballots' counts
    unsigned bal[kRefillOf<T>][4];
    int start[kRefillOf<T>][4];
    int acc = 0;
#pragma unroll
    for (int c = 0; c < 4; c++)
#pragma unroll
      for (int q = 0; q < kRefillOf<T>; q++) {
        bal[q][c] = __ballot_sync(0xffffffffu, cls_q[q] == c);
        start[q][c] = acc;
        acc += __popc(bal[q][c]);
      }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int q = 0; q < kRefillOf<T>; q++) {
      const int c = cls_q[q];
      const unsigned b = c == 0 ? bal[q][0] : c == 1 ? bal[q][1] : c == 2 ? bal[q][2] : bal[q][3];
      const int s0 =
          c == 0 ? start[q][0] : c == 1 ? start[q][1] : c == 2 ? start[q][2] : start[q][3];
      s_dord[wid][s0 + __popc(b & lt)] = (short)(c == 3 ? -1 : q * 32 + lane);
    }
    int ref[3] = {0, 0, 0};
    if (r0 < nvalid) {
#pragma unroll
      for (int l = 0; l < D; l++) ref[l] = pv.cell[l * pv.cap + c0 + r0];
    }
    T *win_warp = s_win + (size_t)wid * WarpWin<D>::NE * 32;
    T *win_col = win_warp + lane;
    for (int e = 0; e < WarpWin<D>::NE; e++) win_col[e * 32] = T(0);
    __syncwarp();
    T dtdx[3];
#pragma unroll
    for (int l = 0; l < 3; l++) dtdx[l] = l < D ? kc.dt * ms.inv_dx[l] : T(0);
    if constexpr (!FINAL && std::is_same<S, float>::value) {
      // plain passes of FP32 contexts (their records always exist): every
      // round's record is loaded up front, in the class order, so that the
      // range's loads are in flight together (slot -1: an empty slot or a
      // failed particle)
      constexpr int Q = kRefillOf<T>;
      float4 ra[Q], rb[Q];
      int kq[Q];
#pragma unroll
      for (int q = 0; q < Q; q++) {
        kq[q] = q < nr ? s_dord[wid][q * 32 + lane] : -1;
        if (kq[q] >= 0) {
          const int64_t i = c0 + r0 + kq[q];
          ra[q] = rec[2 * i];
          rb[q] = rec[2 * i + 1];
        }
      }
#pragma unroll 1
      for (int q = 0; q < nr; q++) {
        const float4 a = ra[0], b = rb[0];
        const int k0 = kq[0];
#pragma unroll
        for (int t = 0; t + 1 < Q; t++) {
          ra[t] = ra[t + 1];
          rb[t] = rb[t + 1];
          kq[t] = kq[t + 1];
        }
        if (k0 >= 0) {
          DepIn<T> cur;
          dep_from_rec<D, T>(cur, a, b);
          PushConst<T> pc;
          pc.q = cur.q;
          deposit_orbit<D, T, FINAL, false>(pc, cur.cell, cur.off, dtdx, T(0), T(1), kc.dt, T(1),
                                            cur.vb, nodes, nodes_u, J, pg, kc, ms, win_col, ref,
                                            npieces, st, work, chain, 2);
        }
      }
    } else {
    // the deposits; each round's particle data is loaded one round ahead
    // (slot -1: an empty slot or a failed particle)
    DepIn<T> cur, nxt;
    int kcur = s_dord[wid][lane];
    if (kcur >= 0) dep_load<D, T, S>(cur, pv, c0 + r0 + kcur, kc, rec);
#pragma unroll 1
    for (int q = 0; q < nr; q++) {
      const int knx = q + 1 < nr ? s_dord[wid][(q + 1) * 32 + lane] : -1;
      if (knx >= 0) dep_load<D, T, S>(nxt, pv, c0 + r0 + knx, kc, rec);
      if (kcur >= 0) {
        PushConst<T> pc;
        if (FINAL) {  // the work and chain-rule sums need the push constants
          LaneSolve<D, T> d;
          lane_init<D, T, S>(d, pv, c0 + r0 + kcur, kc, ms);
          pc = d.pc;
        } else {
          pc.q = cur.q;
        }
        deposit_orbit<D, T, FINAL, false>(pc, cur.cell, cur.off, dtdx, T(0), T(1), kc.dt, T(1),
                                          cur.vb, nodes, nodes_u, J, pg, kc, ms, win_col, ref,
                                          npieces, st, work, chain, 2);
      }
      cur = nxt;
      kcur = knx;
    }
    }
    __syncwarp();
    for (int e = lane; e < WarpWin<D>::NE; e += 32) {
      const T *rowp = win_warp + (size_t)e * 32;
      T sum = T(0);
#pragma unroll 8
      for (int l = 0; l < 32; l++) sum += rowp[(l + lane) & 31];
      if (sum != T(0)) {
        const int node = e / 3, c = e - 3 * node;
        const int rx = node % WarpWin<D>::N0 + WarpWin<D>::LO0;
        const int ry = node / WarpWin<D>::N0 + WarpWin<D>::LO1;
        int g = (ref[0] + rx) & pg.mask[0];
        if (D > 1) g += pg.n0 * ((ref[1] + ry) & pg.mask[1]);
        atomicAdd(J + (size_t)c * pg.Ng + g, widen(sum));
      }
    }
  } else {
    // FP64 and 3D: direct atomics, kPT particles at a time in the order of
    // s_order (given by the caller, else that of the knot planes the final
    // orbits cross)
    __shared__ int s_own[kChunkOf<T>];  // room for the longest chunk
    if (!s_order) {
      s_order = s_own;
      const GSrc<S> src{&pv, pv.vbar};
      order_chunk<D, T>(src, c0, nvalid, kc, ms, s_order);
    }
#pragma unroll 1
    for (int q = 0; q < nr; q++) {
      const int kk = q * kPT + threadIdx.x;
      const int64_t ip = kk < nvalid ? c0 + s_order[kk] : -1;
      if (ip >= 0 && pv.iters[ip] > 0) {
        LaneSolve<D, T> d;
        lane_init<D, T, S>(d, pv, ip, kc, ms);
#pragma unroll
        for (int c = 0; c < 3; c++) d.vb[c] = (T)pv.vbar[c * pv.cap + ip];
        const int ref[3] = {0, 0, 0};
        deposit_orbit<D, T, FINAL, false>(d.pc, d.cell, d.off, d.dtdx, T(0), T(1), kc.dt, T(1),
                                          d.vb, nodes, nodes_u, J, pg, kc, ms, nullptr, ref,
                                          npieces, st, work, chain, 2);
      }
    }
  }
  if (st) atomicOr(&cnt->status, st);
  const unsigned pc_w = __reduce_add_sync(0xffffffffu, (unsigned)npieces);
  if (lane == 0) atomicAdd(&cnt->pieces, (unsigned long long)pc_w);
}

// FP32 instances: at least 4 resident CTAs (<= 128 registers) to hide latency;
// FP64 instances are bound by the FP64 pipe and keep their registers.
// S is the particle storage type: T itself, or double under FP32 arithmetic
// (the FP32 stage of an FP64 context, option fp32_first).
// tim (may be null): the launch's first CTA start and last CTA end on the
// global nanosecond timer, folded in with atomicMin / atomicMax (device-side
// timing for launches inside a graph loop, where events cannot accumulate).
template <int D, typename T, bool FINAL, bool GEN, typename S = T>
__global__ void __launch_bounds__(kPT, sizeof(T) == 4 ? 4 : 1)
k_map(PView<S> pv, const T *__restrict__ nodes, const T *__restrict__ nodes_u,
      double *__restrict__ J, PGeom pg, KConst<T> kc, EvalCounters *__restrict__ cnt,
      double *__restrict__ psum, unsigned long long *__restrict__ tim) {
  if (tim && threadIdx.x == 0) atomicMin(tim, global_ns());
  const MapScale<T> ms = {{kc.inv_dx[0], kc.inv_dx[1], kc.inv_dx[2]}, kc.inv_dV};
  map_block<D, T, FINAL, GEN, S>(pv, blockIdx.x * (int64_t)kPT + threadIdx.x, nodes, nodes_u, J,
                                 pg, kc, ms, cnt, psum + 2 * (size_t)blockIdx.x);
  if (tim) {
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(tim + 1, global_ns());
  }
}

// The FP32 solve launch stages each chunk's inputs in shared memory (dynamic
// shared memory of Stage<D, float>::kBytes); FP64 and the FP32 stage of FP64
// contexts read them from global memory.
template <typename T, typename S>
constexpr bool kStaged = std::is_same<T, float>::value && std::is_same<S, float>::value;

// The common path (quadratic shapes, no refinement, FP64 or FP32 arithmetic)
// as two launches over chunks of nr * kPT particles (nr <= kRefillOf<T>,
// chosen by the host for the problem size): the inner solves with lane
// refill, then the deposits.  Two kernels rather than one keep each kernel's
// code small and let the deposit pass start on a chunk without waiting at a
// barrier for the chunk's slowest inner solve.  tim as for k_map: the solve
// launch records the start, the deposit launch the end.
template <int D, typename T, typename S = T>
__global__ void __launch_bounds__(kPT, sizeof(T) == 4 ? 4 : 1)
k_map_solve(PView<S> pv, const T *__restrict__ nodes, PGeom pg, KConst<T> kc,
            EvalCounters *__restrict__ cnt, unsigned long long *__restrict__ tim, int nr) {
  if (tim && threadIdx.x == 0) atomicMin(tim, global_ns());
  const MapScale<T> ms = {{kc.inv_dx[0], kc.inv_dx[1], kc.inv_dx[2]}, kc.inv_dV};
  __shared__ int s_order[kChunkOf<T>];
  if constexpr (kStaged<T, S>) {
    extern __shared__ __align__(16) char s_stage[];  // Stage<D, S>::kBytes
    __shared__ unsigned long long s_bar;
    map_chunk_solve<D, T, S>(pv, blockIdx.x * (int64_t)(nr * kPT), nodes, pg, kc, ms, cnt,
                             s_order, s_stage, &s_bar, nr);
  } else {
    map_chunk_solve<D, T, S>(pv, blockIdx.x * (int64_t)(nr * kPT), nodes, pg, kc, ms, cnt,
                             s_order, nullptr, nullptr, nr);
  }
}

template <int D, typename T, bool FINAL, typename S = T>
__global__ void __launch_bounds__(kPT, sizeof(T) == 4 ? 4 : 1)
k_map_deposit(PView<S> pv, const T *__restrict__ nodes, const T *__restrict__ nodes_u,
              double *__restrict__ J, PGeom pg, KConst<T> kc, EvalCounters *__restrict__ cnt,
              double *__restrict__ psum, unsigned long long *__restrict__ tim, int nr) {
  const MapScale<T> ms = {{kc.inv_dx[0], kc.inv_dx[1], kc.inv_dx[2]}, kc.inv_dV};
  double work = 0.0, chain = 0.0;
  map_chunk_deposit<D, T, FINAL, S>(pv, blockIdx.x * (int64_t)(nr * kPT), nodes, nodes_u, J, pg,
                                    kc, ms, cnt, work, chain, nullptr, nr);
  if (FINAL) {
    double v[2] = {work, chain};
    block_sums<2>(v, psum + 2 * (size_t)blockIdx.x);
  }
  if (tim) {
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(tim + 1, global_ns());
  }
}

// The same two passes in one launch (FP64 arithmetic): the FP64 map is bound
// by the FP64 pipe rather than by latency, so a chunk's deposits follow its
// inner solves in the same CTA, while the particles are still in L2.  The
// grid is persistent (as many CTAs as fit at once): each CTA takes chunks
// from a counter until nchunks are done, so no partial last wave of CTAs
// idles the SMs.  psum[2 c .. 2 c + 2) receives chunk c's final-pass partials.
template <int D, typename T, bool FINAL, typename S = T>
__global__ void __launch_bounds__(kPT, 1)
k_map_fused(PView<S> pv, const T *__restrict__ nodes, const T *__restrict__ nodes_u,
            double *__restrict__ J, PGeom pg, KConst<T> kc, EvalCounters *__restrict__ cnt,
            double *__restrict__ psum, unsigned long long *__restrict__ tim, int nchunks,
            int nr) {
  if (tim && threadIdx.x == 0) atomicMin(tim, global_ns());
  const MapScale<T> ms = {{kc.inv_dx[0], kc.inv_dx[1], kc.inv_dx[2]}, kc.inv_dV};
  __shared__ int s_order[kChunkOf<T>];
  __shared__ int s_chunk;
#pragma unroll 1
  for (;;) {
    if (threadIdx.x == 0) s_chunk = (int)atomicAdd(&cnt->chunk_next, 1u);
    __syncthreads();
    const int ch = s_chunk;
    if (ch >= nchunks) break;
    const int64_t c0 = ch * (int64_t)(nr * kPT);
    map_chunk_solve<D, T, S>(pv, c0, nodes, pg, kc, ms, cnt, s_order, nullptr, nullptr, nr);
    __syncthreads();  // every orbit velocity of the chunk stored
    // the deposits in the solve's order (predicted crossings)
    double work = 0.0, chain = 0.0;
    map_chunk_deposit<D, T, FINAL, S>(pv, c0, nodes, nodes_u, J, pg, kc, ms, cnt, work, chain,
                                      s_order, nr);
    if (FINAL) {  // per-chunk partials: merged in chunk order, whichever CTA ran the chunk
      double v[2] = {work, chain};
      block_sums<2>(v, psum + 2 * (size_t)ch);
    }
    __syncthreads();  // s_order and s_chunk are reused by the next chunk
  }
  if (tim) {
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(tim + 1, global_ns());
  }
}

}  // namespace
