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

// Constants of the particle map in the particle real type, so that the FP32
// instance does no FP64 conversion inside its loops (the FP64 pipe of the
// B300 is 1/64 of the FP32 one).
template <typename T>
struct KConst {
  T dt, kappa, tau_r, tau_a, inv_dV;
  T inv_dx[3];
  T gl_t[PIC_MAX_GL], gl_w[PIC_MAX_GL];
  int ngl, inner_max, warm;
  double qs[PIC_MAX_SPECIES], ms[PIC_MAX_SPECIES];
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
  for (int s = 0; s < PIC_MAX_SPECIES; s++) {
    k.qs[s] = sc.qs[s];
    k.ms[s] = sc.ms[s];
  }
  return k;
}

// Exact widening of a deposit contribution to FP64 for the global atomics.
// For FP32 the conversion is done with integer operations (sign, exponent
// rebias by 1023 - 127 = 896, mantissa shift by 29) so that it does not
// occupy the narrow FP64 pipe; FP32 subnormals (< 1.2e-38) flush to zero.
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  const unsigned hi = (u & 0x80000000u) | ((((u >> 3) & 0x0fffffffu)) + (896u << 20));
  const unsigned lo = u << 29;
  return __hiloint2double((int)hi, (int)lo);
}

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

template <int D, typename T, bool DERIV>
__device__ __forceinline__ void accumulate_piece(const KConst<T> &kc, const T off[3],
                                                 const T del[3], const int base[3], T sa, T sb,
                                                 PieceAcc<D, T> &pa) {
  constexpr int NN = PieceAcc<D, T>::NN;
#pragma unroll
  for (int k = 0; k < NN; k++) {
    pa.Sb[k] = T(0);
#pragma unroll
    for (int j = 0; j < D; j++) pa.Wd[j][k] = pa.W1[j][k] = T(0);
  }
  const T len = sb - sa;
  T t0[3];
#pragma unroll
  for (int l = 0; l < D; l++) t0[l] = off[l] - T(base[l]);
#pragma unroll 1
  for (int qp = 0; qp < kc.ngl; qp++) {
    const T s = sa + len * kc.gl_t[qp];
    const T wt = len * kc.gl_w[qp];
    T S[3][3], dS[3][3];
#pragma unroll
    for (int l = 0; l < D; l++) qspline<T>(t0[l] + s * del[l], S[l], dS[l]);
    if (D == 1) {
#pragma unroll
      for (int i = 0; i < 3; i++) {
        pa.Sb[i] += wt * S[0][i];
        if (DERIV) {
          T b = wt * dS[0][i];
          pa.Wd[0][i] += b;
          pa.W1[0][i] += s * b;
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
          pa.Sb[k] += a * S[1][j];
          if (DERIV) {
            pa.Wd[0][k] += b * S[1][j];
            pa.W1[0][k] += e * S[1][j];
            pa.Wd[D > 1 ? 1 : 0][k] += a * dS[1][j];
            pa.W1[D > 1 ? 1 : 0][k] += c * dS[1][j];
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
            pa.Sb[k] += ab * S[2][l];
            if (DERIV) {
              const T d0 = dab * S[2][l], d1 = adb * S[2][l], d2 = ab * dS[2][l];
              pa.Wd[0][k] += d0;
              pa.W1[0][k] += s * d0;
              pa.Wd[D > 1 ? 1 : 0][k] += d1;
              pa.W1[D > 1 ? 1 : 0][k] += s * d1;
              pa.Wd[D > 2 ? 2 : 0][k] += d2;
              pa.W1[D > 2 ? 2 : 0][k] += s * d2;
            }
          }
        }
    }
  }
}

// 3D: the same orbit integrals for the 9 nodes (ox, oy) of one z-slab oz of
// the 27-node stencil, so that the accumulators of a slab (9 x 7 values) fit
// in registers; the caller loops over the three slabs and contracts each.
template <typename T, bool DERIV>
__device__ __forceinline__ void accumulate_slab(const KConst<T> &kc, const T off[3],
                                                const T del[3], const int base[3], T sa, T sb,
                                                int oz, PieceAcc<2, T> &pa, T (&Wz)[9],
                                                T (&W1z)[9]) {
#pragma unroll
  for (int k = 0; k < 9; k++) {
    pa.Sb[k] = T(0);
    pa.Wd[0][k] = pa.W1[0][k] = pa.Wd[1][k] = pa.W1[1][k] = T(0);
    Wz[k] = W1z[k] = T(0);
  }
  const T len = sb - sa;
  T t0[3];
#pragma unroll
  for (int l = 0; l < 3; l++) t0[l] = off[l] - T(base[l]);
#pragma unroll 1
  for (int qp = 0; qp < kc.ngl; qp++) {
    const T s = sa + len * kc.gl_t[qp];
    const T wt = len * kc.gl_w[qp];
    T S[3][3], dS[3][3];
#pragma unroll
    for (int l = 0; l < 3; l++) qspline<T>(t0[l] + s * del[l], S[l], dS[l]);
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

// Inner-iteration gather: grad phi-bar (Eq. orbit-gather-general with
// G = grad phi^{1/2}) and the discrete gradient D (3 x D, node units until
// the caller scales column j by 1/dx_j).
template <int D, typename T>
struct GatherOrbit {
  const T *__restrict__ nodes;
  const PGeom *pg;
  const KConst<T> *kc;
  int cell[3];
  T off[3], del[3];
  T gphi[3];
  T Dm[3][3];
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
        accumulate_slab<T, true>(*kc, off, del, base, sa, sb, oz, pa, Wz, W1z);
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
#pragma unroll
            for (int c = 0; c < 3; c++) {
              const T An = r[D + c], dA = r[D + 3 + c] - An;
              Dm[c][0] += An * pa.Wd[0][k] + dA * pa.W1[0][k];
              Dm[c][1] += An * pa.Wd[1][k] + dA * pa.W1[1][k];
              Dm[c][D > 2 ? 2 : 0] += An * Wz[k] + dA * W1z[k];
            }
          }
      }
      return;
    }
    PieceAcc<D, T> pa;
    accumulate_piece<D, T, true>(*kc, off, del, base, sa, sb, pa);
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
#pragma unroll
          for (int c = 0; c < 3; c++) {
            const T An = r[D + c], dA = r[D + 3 + c] - An;
#pragma unroll
            for (int j = 0; j < D; j++) Dm[c][j] += An * pa.Wd[j][k] + dA * pa.W1[j][k];
          }
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
template <int D, typename T, bool FINAL>
struct DepositOrbit {
  const T *__restrict__ nodes;
  const T *__restrict__ nodes_u;
  double *__restrict__ J;
  const PGeom *pg;
  const KConst<T> *kc;
  int cell[3];
  T off[3], del[3];
  T qv[3];  // q vbar / dV
  T gphi[3], Ubar[3], Dm[3][3];
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
        accumulate_slab<T, FINAL>(*kc, off, del, base, sa, sb, oz, pa, Wz, W1z);
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
              for (int c = 0; c < 3; c++) {
                Ubar[c] += u[c] * pa.Sb[k];
                const T An = r[D + c], dA = r[D + 3 + c] - An;
                Dm[c][0] += An * pa.Wd[0][k] + dA * pa.W1[0][k];
                Dm[c][1] += An * pa.Wd[1][k] + dA * pa.W1[1][k];
                Dm[c][D > 2 ? 2 : 0] += An * Wz[k] + dA * W1z[k];
              }
            }
#pragma unroll
            for (int c = 0; c < 3; c++)
              atomicAdd(J + (size_t)c * pg->Ng + g, widen(qv[c] * pa.Sb[k]));
          }
      }
      return;
    }
    PieceAcc<D, T> pa;
    accumulate_piece<D, T, FINAL>(*kc, off, del, base, sa, sb, pa);
    // window coordinates of the piece's base node (relative to ref)
    int wx = 0, wy = 0;
    if (WarpWin<D>::kOn && win) {
      wx = wrap_rel(cell[0] + base[0] - ref[0], pg->n[0]) - 1 - WarpWin<D>::LO0;
      wy = D > 1 ? wrap_rel(cell[1] + base[1] - ref[1], pg->n[1]) - 1 - WarpWin<D>::LO1 : 0;
    }
#pragma unroll
    for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
#pragma unroll
      for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
#pragma unroll
        for (int ox = 0; ox < 3; ox++) {
          const int k = ox + 3 * (oy + 3 * oz);
          const int g = nr.at(ox, oy, oz);
          if (FINAL) {
            T r[NVP], u[4];
            load_rec<NVP>(nodes + (size_t)g * NVP, r);
            load_rec<4>(nodes_u + (size_t)g * 4, u);
#pragma unroll
            for (int c = 0; c < D; c++) gphi[c] += r[c] * pa.Sb[k];
#pragma unroll
            for (int c = 0; c < 3; c++) {
              Ubar[c] += u[c] * pa.Sb[k];
              const T An = r[D + c], dA = r[D + 3 + c] - An;
#pragma unroll
              for (int j = 0; j < D; j++) Dm[c][j] += An * pa.Wd[j][k] + dA * pa.W1[j][k];
            }
          }
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
            else atomicAdd(J + (size_t)c * pg->Ng + g, widen(v));
          }
        }
  }
};

// A^{n+1}_h at u = off + del (node coordinates relative to the cell) from the
// node records (Eq. mesh-interpolant)
template <int D, typename T>
__device__ __forceinline__ void interp_A1(const PGeom &pg, const int cell[3], const T u[3],
                                          const T *__restrict__ nodes, T out[3]) {
  constexpr int NVP = Rec<D>::NVP;
  int base[3] = {0, 0, 0};
  T Sw[3][3];
#pragma unroll
  for (int l = 0; l < D; l++) {
    base[l] = (int)floor(u[l] + T(0.5));
    qspline_val<T>(u[l] - T(base[l]), Sw[l]);
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

// A_h(u) from a component-major FP64 mesh array (step start, energy, deposits)
template <int D, typename T>
__device__ __forceinline__ void point_interp(const PGeom &pg, const int cell[3], const T u[3],
                                             const double *__restrict__ F, T out[3]) {
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

// FP32 instances: at least 4 resident CTAs (<= 128 registers) to hide latency;
// FP64 instances are bound by the FP64 pipe and keep their registers
template <int D, typename T, bool FINAL>
__global__ void __launch_bounds__(kPT, sizeof(T) == 4 ? 4 : 1)
k_map(PView<T> pv, const T *__restrict__ nodes, const T *__restrict__ nodes_u,
      double *__restrict__ J, PGeom pg, KConst<T> kc, EvalCounters *__restrict__ cnt,
      double *__restrict__ psum) {
  const int64_t i = blockIdx.x * (int64_t)kPT + threadIdx.x;
  const bool active = i < pv.np;
  double work = 0.0, chain = 0.0;
  int iters = 0, npieces = 0;
  unsigned int st = 0;
  // FP32 deposit window of this warp (see WarpWin): reference cell = the
  // cell of the warp's first particle, columns zeroed by their lanes
  constexpr bool kWin = WarpWin<D>::kOn && sizeof(T) == 4;
  __shared__ T s_win[kWin ? (kPT / 32) * WarpWin<D>::NE * 32 : 1];
  T *win_warp = s_win + (size_t)(threadIdx.x >> 5) * WarpWin<D>::NE * 32;
  T *win_col = kWin ? win_warp + (threadIdx.x & 31) : nullptr;
  int ref[3] = {0, 0, 0};
  if (kWin) {
    const int64_t i0 = i - (threadIdx.x & 31);  // the warp's first particle
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
      off[l] = pv.off[l * cap + i];
      dtdx[l] = dt * kc.inv_dx[l];
    }
    T vb[3], Pn1[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      pc.Pn[c] = pv.P[c * cap + i];
      pc.Am[c] = pv.Am[c * cap + i];
      pc.pn[c] = pc.Pn[c] - pc.q * pc.Am[c];
      vb[c] = kc.warm ? pv.vbar[c * cap + i] : pv.v0[c * cap + i];
      Pn1[c] = pc.Pn[c];
    }
    pc.gamma_n = sqrt(T(1) + (pc.pn[0] * pc.pn[0] + pc.pn[1] * pc.pn[1] + pc.pn[2] * pc.pn[2]) *
                                 pc.inv_mk * pc.inv_mk);
    const T tau_r = kc.tau_r, tau_a = kc.tau_a, kap2 = kap * kap;
    bool conv = false;
    int it;
#pragma unroll 1
    for (it = 1; it <= kc.inner_max; it++) {
      GatherOrbit<D, T> go;
      go.nodes = nodes;
      go.pg = &pg;
      go.kc = &kc;
      go.pieces = 0;
#pragma unroll
      for (int l = 0; l < 3; l++) {
        go.cell[l] = cell[l];
        go.off[l] = off[l];
        go.del[l] = vb[l] * dtdx[l];
        go.gphi[l] = T(0);
        go.Dm[l][0] = go.Dm[l][1] = go.Dm[l][2] = T(0);
      }
      const bool ok = walk_orbit<D, T>(go.off, go.del, go);
      npieces += go.pieces;
      if (!ok) {
        st |= PIC_ST_PIECES;
        break;
      }
#pragma unroll
      for (int c = 0; c < 3; c++)
#pragma unroll
        for (int j = 0; j < D; j++) go.Dm[c][j] *= kc.inv_dx[j];
      T u1[3], Ap[3];
#pragma unroll
      for (int l = 0; l < 3; l++) u1[l] = go.off[l] + go.del[l];
      interp_A1<D, T>(pg, cell, u1, nodes, Ap);
      T vn[3], Pc[3];
      gmhc_push<D, T>(pc, Ap, go.gphi, go.Dm, vb, vn, Pc);
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
      if (v2 >= kap2) { st |= PIC_ST_SUPERLUM; break; }
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
      const T qdv = pc.q * kc.inv_dV;
      DepositOrbit<D, T, FINAL> dp;
      dp.nodes = nodes;
      dp.nodes_u = nodes_u;
      dp.J = J;
      dp.pg = &pg;
      dp.kc = &kc;
      dp.pieces = 0;
      dp.win = win_col;
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
      if (!walk_orbit<D, T>(dp.off, dp.del, dp)) st |= PIC_ST_PIECES;
      npieces += dp.pieces;
      if (FINAL) {
        T u1[3], Ap[3];
#pragma unroll
        for (int l = 0; l < 3; l++) u1[l] = dp.off[l] + dp.del[l];
        interp_A1<D, T>(pg, cell, u1, nodes, Ap);
#pragma unroll
        for (int c = 0; c < 3; c++) {
          T Dv = T(0);
#pragma unroll
          for (int j = 0; j < D; j++) Dv += dp.Dm[c][j] * kc.inv_dx[j] * vb[j];
          T Eb = -(c < D ? dp.gphi[c] : T(0)) - dp.Ubar[c];
          work += (double)(pc.q * vb[c] * Eb);
          T RA = Ap[c] - pc.Am[c] - dt * (dp.Ubar[c] + Dv);
          chain += (double)RA * (double)RA;
        }
      }
    }
  }
  if (kWin) {
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
  const int mx = __reduce_max_sync(0xffffffffu, iters);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&cnt->inner_sum, (unsigned long long)it_sum);
    atomicAdd(&cnt->pieces, (unsigned long long)pc_sum);
    if (mx > 0) atomicMax(&cnt->inner_max, mx);
  }
  if (FINAL) {
    double v[2] = {work, chain};
    block_sums<2>(v, psum);
  }
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
  point_interp<D, double>(pg, cell, off, A, Ax);
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
  point_interp<D, double>(pg, cell, off, A, Ax);
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

// step start: A^- = A^n_h(x^n), p^n = P^n - q A^-, v^0 = v(p^n),
// in the particle real type; AT is A^n in that type (component-major)
template <int D, typename T>
__global__ void k_step_start(PView<T> pv, T *Am, T *v0, T *vbar, const T *__restrict__ AT,
                             PGeom pg, KConst<T> kc) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= pv.np) return;
  int cell[3] = {0, 0, 0};
  T off[3] = {T(0), T(0), T(0)};
  for (int l = 0; l < D; l++) {
    cell[l] = pv.cell[l * pv.cap + i];
    off[l] = pv.off[l * pv.cap + i];
  }
  T Ax[3];
  point_interp_T<D, T>(pg, cell, off, AT, Ax);
  int s = pv.sp[i];
  T q = (T)(pv.w[i] * kc.qs[s]), m = (T)(pv.w[i] * kc.ms[s]);
  T p[3], p2 = T(0);
  for (int c = 0; c < 3; c++) {
    Am[c * pv.cap + i] = Ax[c];
    p[c] = pv.P[c * pv.cap + i] - q * Ax[c];
    p2 += p[c] * p[c];
  }
  const T im = T(1) / m, ik = T(1) / kc.kappa;
  T ig = rsqrt(T(1) + p2 * im * im * ik * ik);
  for (int c = 0; c < 3; c++) {
    const T v = p[c] * im * ig;
    v0[c * pv.cap + i] = v;
    vbar[c * pv.cap + i] = v;  // warm starts of the step begin from v(p^n) too
  }
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
// (Eq. Kkin-nondim): per particle in the particle real type, summed in that
// type over a warp and in FP64 from there on (block partials summed on the host)
template <int D, typename T>
__global__ void __launch_bounds__(kPT)
k_kinetic(PView<T> pv, const T *__restrict__ AT, PGeom pg, KConst<T> kc, double *psum) {
  int64_t i = blockIdx.x * (int64_t)kPT + threadIdx.x;
  T k = T(0);
  if (i < pv.np) {
    int cell[3] = {0, 0, 0};
    T off[3] = {T(0), T(0), T(0)};
    for (int l = 0; l < D; l++) {
      cell[l] = pv.cell[l * pv.cap + i];
      off[l] = pv.off[l * pv.cap + i];
    }
    T Ax[3];
    point_interp_T<D, T>(pg, cell, off, AT, Ax);
    int s = pv.sp[i];
    T q = (T)(pv.w[i] * kc.qs[s]), m = (T)(pv.w[i] * kc.ms[s]);
    T p2 = T(0);
    for (int c = 0; c < 3; c++) {
      T p = pv.P[c * pv.cap + i] - q * Ax[c];
      p2 += p * p;
    }
    const T im = T(1) / m;
    T gam = sqrt(T(1) + p2 * im * im / (kc.kappa * kc.kappa));
    k = p2 * im / (gam + T(1));
  }
  for (int o = 16; o > 0; o >>= 1) k += __shfl_down_sync(0xffffffffu, k, o);
  __shared__ double sh[kPT / 32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = widen(k);
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kPT / 32; w++) t += sh[w];
    psum[blockIdx.x] = t;
  }
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
                   (void **)&ctx->tmp_i, (void **)&ctx->psum, (void **)&ctx->keys,
                   (void **)&ctx->tmp_l};
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
  CK(cudaMalloc((void **)&ctx->keys, sizeof(int32_t) * cap));
  CK(cudaMalloc((void **)&ctx->tmp_l, sizeof(int64_t) * cap));
  CK(cudaMalloc((void **)&ctx->psum, sizeof(double) * 4 * nb + 64));
  if (ctx->psum_host) cudaFreeHost(ctx->psum_host);
  ctx->psum_host = nullptr;
  CK(cudaMallocHost((void **)&ctx->psum_host, sizeof(double) * 4 * nb + 64));
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

// A^n in the particle real type: the FP64 path reads A_real directly, the
// mixed path a float copy refreshed by particles_refresh_A
template <typename T>
const T *A_typed(pic_ctx *ctx);
template <>
const double *A_typed<double>(pic_ctx *ctx) { return ctx->A_real; }
template <>
const float *A_typed<float>(pic_ctx *ctx) { return (const float *)ctx->A_real_f; }

int particles_step_start(pic_ctx *ctx) {
  if (ctx->np == 0) return PIC_OK;
  PGeom pg = pgeom(ctx);
  StepConst sc = base_sc(ctx);
  PIC_DISPATCH(ctx, (k_step_start<DD, RT><<<nblk(ctx->np), kPT, 0, ctx->st>>>(
                         pview<RT>(ctx), (RT *)ctx->Am, (RT *)ctx->v0, (RT *)ctx->vbar,
                         A_typed<RT>(ctx), pg, kconst<RT>(sc, pg))));
  KCHECK();
  return PIC_OK;
}

int particles_map_launch(pic_ctx *ctx, const StepConst &sc_in, int final_pass) {
  CK(cudaMemsetAsync(ctx->cnt_dev, 0, sizeof(EvalCounters), ctx->st));
  int nb = nblk(ctx->np);
  ctx->map_final = final_pass;
  if (ctx->np > 0) {
    PGeom pg = pgeom(ctx);
    // inside a stream capture the records must become event nodes of the graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(ctx->st, &cap));
    const unsigned evf = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    CK(cudaEventRecordWithFlags(ctx->ev0, ctx->st, evf));
    if (final_pass)
      PIC_DISPATCH(ctx, (k_map<DD, RT, true><<<nb, kPT, 0, ctx->st>>>(
                             pview<RT>(ctx), (const RT *)ctx->nodes, (const RT *)ctx->nodes_u,
                             ctx->Jorb, pg, kconst<RT>(sc_in, pg), ctx->cnt_dev, ctx->psum)));
    else
      PIC_DISPATCH(ctx, (k_map<DD, RT, false><<<nb, kPT, 0, ctx->st>>>(
                             pview<RT>(ctx), (const RT *)ctx->nodes, (const RT *)ctx->nodes_u,
                             ctx->Jorb, pg, kconst<RT>(sc_in, pg), ctx->cnt_dev, ctx->psum)));
    KCHECK();
    CK(cudaEventRecordWithFlags(ctx->ev1, ctx->st, evf));
    if (final_pass)  // block partials of the work and chain-rule sums
      CK(cudaMemcpyAsync(ctx->psum_host, ctx->psum, sizeof(double) * 2 * nb,
                         cudaMemcpyDeviceToHost, ctx->st));
  }
  CK(cudaMemcpyAsync(ctx->cnt_host, ctx->cnt_dev, sizeof(EvalCounters), cudaMemcpyDeviceToHost,
                     ctx->st));
  return PIC_OK;
}

int particles_map_finish(pic_ctx *ctx, double *work_sum, double *chain_sum, EvalCounters *cnt) {
  double work = 0.0, chain = 0.0;
  if (ctx->np > 0) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    ctx->map_ms += ms;
    ctx->map_launches++;
    if (ctx->map_final) {  // fixed summation order: reproducible diagnostics
      int nb = nblk(ctx->np);
      for (int b = 0; b < nb; b++) {
        work += ctx->psum_host[2 * b];
        chain += ctx->psum_host[2 * b + 1];
      }
    }
  }
  *cnt = *ctx->cnt_host;
  ctx->pushes += ctx->np;
  ctx->inner_iters += (long long)cnt->inner_sum;
  ctx->pieces += (long long)cnt->pieces;
  if (work_sum) *work_sum = work;
  if (chain_sum) *chain_sum = chain;
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
  PIC_DISPATCH(ctx, (k_kinetic<DD, RT><<<nb, kPT, 0, ctx->st>>>(
                         pview<RT>(ctx), A_typed<RT>(ctx), pg, kconst<RT>(sc, pg), ctx->psum)));
  KCHECK();
  CK(cudaMemcpyAsync(ctx->psum_host, ctx->psum, sizeof(double) * nb, cudaMemcpyDeviceToHost,
                     ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  double k = 0.0;
  for (int b = 0; b < nb; b++) k += ctx->psum_host[b];  // fixed order
  *K = k;
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

__global__ void k_to_float(const double *__restrict__ a, float *__restrict__ b, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

int particles_refresh_A(pic_ctx *ctx) {
  if (ctx->rsize == 8) return PIC_OK;
  size_t n = (size_t)3 * ctx->g.Ng;
  k_to_float<<<(unsigned)((n + 255) / 256), 256, 0, ctx->st>>>(ctx->A_real, (float *)ctx->A_real_f,
                                                               n);
  KCHECK();
  return PIC_OK;
}

// ---- counting sort of the particles by cell --------------
// key = linear index of the nearest node; a histogram, an exclusive scan and
// a scatter give every particle its slot, and each SoA array is permuted
// through scratch.  The order inside a cell follows the atomic cursor, so it
// is not reproducible from run to run; nothing depends on it except the
// summation order of the deposit (the load-order index restores the caller's
// order on export).
__global__ void k_sort_keys(int64_t np, int64_t cap, const int32_t *__restrict__ cell, int dim,
                            int n0, int n01, int32_t *__restrict__ keys,
                            int32_t *__restrict__ count) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  int k = cell[i];
  if (dim > 1) k += n0 * cell[cap + i];
  if (dim > 2) k += n01 * cell[2 * cap + i];
  keys[i] = k;
  atomicAdd(count + k, 1);
}

// exclusive scan of count[0, Ng) in place (one block of 1024 threads)
__global__ void k_sort_scan(int32_t *count, int Ng) {
  __shared__ int32_t sh[1024];
  const int chunk = (Ng + 1023) / 1024;
  const int t0 = threadIdx.x * chunk;
  int32_t s = 0;
  for (int k = t0; k < min(t0 + chunk, Ng); k++) s += count[k];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
    int32_t v = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  int32_t run = sh[threadIdx.x] - s;  // exclusive prefix of this chunk
  for (int k = t0; k < min(t0 + chunk, Ng); k++) {
    int32_t c = count[k];
    count[k] = run;
    run += c;
  }
}

__global__ void k_sort_slots(int64_t np, const int32_t *__restrict__ keys, int32_t *cursor,
                             int64_t *__restrict__ slot) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  slot[i] = atomicAdd(cursor + keys[i], 1);
}

template <typename V>
__global__ void k_permute(int64_t np, int64_t cap, int ncomp, const V *__restrict__ src,
                          V *__restrict__ dst, const int64_t *__restrict__ slot) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  int64_t j = slot[i];
  for (int c = 0; c < ncomp; c++) dst[c * cap + j] = src[c * cap + i];
}

template <typename V>
int permute_field(pic_ctx *ctx, V *field, int ncomp) {
  V *scr = (V *)ctx->tmp_d;  // 7 * cap doubles of scratch >= 3 * cap * sizeof(V)
  k_permute<V><<<nblk(ctx->np), kPT, 0, ctx->st>>>(ctx->np, ctx->cap, ncomp, field, scr,
                                                   ctx->tmp_l);
  KCHECK();
  for (int c = 0; c < ncomp; c++)
    CK(cudaMemcpyAsync(field + (size_t)c * ctx->cap, scr + (size_t)c * ctx->cap,
                       sizeof(V) * ctx->np, cudaMemcpyDeviceToDevice, ctx->st));
  return PIC_OK;
}

int particles_sort(pic_ctx *ctx) {
  if (ctx->np < 2) return PIC_OK;
  const Geom &g = ctx->g;
  CK(cudaMemsetAsync(ctx->cnt_sort, 0, sizeof(int32_t) * g.Ng, ctx->st));
  k_sort_keys<<<nblk(ctx->np), kPT, 0, ctx->st>>>(ctx->np, ctx->cap, ctx->cell, g.dim, g.n[0],
                                                  g.n[0] * g.n[1], ctx->keys, ctx->cnt_sort);
  KCHECK();
  k_sort_scan<<<1, 1024, 0, ctx->st>>>(ctx->cnt_sort, g.Ng);
  KCHECK();
  k_sort_slots<<<nblk(ctx->np), kPT, 0, ctx->st>>>(ctx->np, ctx->keys, ctx->cnt_sort, ctx->tmp_l);
  KCHECK();
  int e;
  if ((e = permute_field<int32_t>(ctx, ctx->cell, g.dim))) return e;
  if (ctx->rsize == 8) {
    if ((e = permute_field<double>(ctx, (double *)ctx->off, g.dim))) return e;
    if ((e = permute_field<double>(ctx, (double *)ctx->P, 3))) return e;
  } else {
    if ((e = permute_field<float>(ctx, (float *)ctx->off, g.dim))) return e;
    if ((e = permute_field<float>(ctx, (float *)ctx->P, 3))) return e;
  }
  if ((e = permute_field<double>(ctx, ctx->w, 1))) return e;
  if ((e = permute_field<int32_t>(ctx, ctx->sp, 1))) return e;
  if ((e = permute_field<int64_t>(ctx, ctx->id, 1))) return e;
  CK(cudaStreamSynchronize(ctx->st));
  return PIC_OK;
}
