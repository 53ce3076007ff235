// adjoint_device.cuh -- device helpers shared by the adjoint of a map
// evaluation (adjoint.cu) and of a step (step_adjoint.cu): the deposit's
// transpose as an orbit gather (OrbitDot), the gather's transpose as orbit
// scatters (ScatterOrbit, scatter_A1), the 3 x 3 adjoint solve, and the
// particle's push constants in plain and dual form.
#pragma once
#include "map_device.cuh"

namespace {

// The orbit gather of a component-major mesh vector field with the
// deposit's weights Sbar along the knot-split orbit (the transpose of
// DepositOrbit's deposit).
template <int D, typename T>
struct OrbitDot {
  const double *__restrict__ F;  // 3 x Ng
  const PGeom *pg;
  const KConst<T> *kc;
  int cell[3];
  T off[3], del[3];
  T G[3];
  int order;
  __device__ __forceinline__ void operator()(const int base[3], T sa, T sb) {
    const NodeRows<D> nr(*pg, cell, base);
    const size_t Ng = (size_t)pg->Ng;
    if (D == 3) {
#pragma unroll 1
      for (int oz = 0; oz < 3; oz++) {
        PieceAcc<2, T> pa;
        T Wz[9], W1z[9];
        accumulate_slab<T, false>(*kc, off, del, base, sa, sb, oz, pa, Wz, W1z, order);
        for (int oy = 0; oy < 3; oy++)
          for (int ox = 0; ox < 3; ox++) {
            const int k = ox + 3 * oy, g = nr.at(ox, oy, oz);
            for (int c = 0; c < 3; c++) G[c] += T(F[c * Ng + g]) * pa.Sb[k];
          }
      }
      return;
    }
    PieceAcc<D, T> pa;
    accumulate_piece<D, T, false>(*kc, off, del, base, sa, sb, pa, order);
    for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
      for (int ox = 0; ox < 3; ox++) {
        const int k = ox + 3 * oy, g = nr.at(ox, oy, 0);
        for (int c = 0; c < 3; c++) G[c] += T(F[c * Ng + g]) * pa.Sb[k];
      }
  }
};

// The transpose of GatherOrbit with respect to the records that depend on
// the trial current: the cotangents gphi of the orbit-averaged grad phi^{1/2}
// and gD1 of the raw D_i A sums (their A^{n+1} part, weights W1) scattered to
// Fbar = [grad phi slots (D), A^{n+1} (3)] x Ng.
template <int D>
struct ScatterOrbit {
  double *__restrict__ Fbar;
  const PGeom *pg;
  const KConst<double> *kc;
  int cell[3];
  double off[3], del[3];
  double gphi[3], gD1[3][3];
  int order;
  __device__ __forceinline__ void operator()(const int base[3], double sa, double sb) {
    const NodeRows<D> nr(*pg, cell, base);
    const size_t Ng = (size_t)pg->Ng;
    if (D == 3) {
#pragma unroll 1
      for (int oz = 0; oz < 3; oz++) {
        PieceAcc<2, double> pa;
        double Wz[9], W1z[9];
        accumulate_slab<double, true>(*kc, off, del, base, sa, sb, oz, pa, Wz, W1z, order);
        for (int oy = 0; oy < 3; oy++)
          for (int ox = 0; ox < 3; ox++) {
            const int k = ox + 3 * oy, g = nr.at(ox, oy, oz);
            for (int c = 0; c < D; c++) atomicAdd(Fbar + c * Ng + g, pa.Sb[k] * gphi[c]);
            for (int c = 0; c < 3; c++)
              atomicAdd(Fbar + (D + c) * Ng + g,
                        pa.W1[0][k] * gD1[c][0] + pa.W1[1][k] * gD1[c][1] + W1z[k] * gD1[c][2]);
          }
      }
      return;
    }
    PieceAcc<D, double> pa;
    accumulate_piece<D, double, true>(*kc, off, del, base, sa, sb, pa, order);
    for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
      for (int ox = 0; ox < 3; ox++) {
        const int k = ox + 3 * oy, g = nr.at(ox, oy, 0);
        for (int c = 0; c < D; c++) atomicAdd(Fbar + c * Ng + g, pa.Sb[k] * gphi[c]);
        for (int c = 0; c < 3; c++) {
          double v = 0.0;
          for (int j = 0; j < D; j++) v += pa.W1[j][k] * gD1[c][j];
          atomicAdd(Fbar + (D + c) * Ng + g, v);
        }
      }
  }
};

// transpose of interp_A1: A^{n+1} at the orbit's end point u
template <int D>
__device__ void scatter_A1(const PGeom &pg, const int cell[3], const double u[3],
                           const double gAp[3], double *Fbar, int order) {
  int base[3] = {0, 0, 0};
  double Sw[3][3];
  for (int l = 0; l < D; l++) {
    base[l] = (int)floor(u[l] + 0.5);
    spline_val<double>(order, u[l] - double(base[l]), Sw[l]);
  }
  const NodeRows<D> nr(pg, cell, base);
  const size_t Ng = (size_t)pg.Ng;
  for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
    for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
      for (int ox = 0; ox < 3; ox++) {
        const int g = nr.at(ox, oy, oz);
        const double w = Sw[0][ox] * (D > 1 ? Sw[1][oy] : 1.0) * (D > 2 ? Sw[2][oz] : 1.0);
        for (int c = 0; c < 3; c++) atomicAdd(Fbar + (D + c) * Ng + g, w * gAp[c]);
      }
}

// solve (I - J^T) x = b for 3 x 3 J by Cramer's rule; false if singular
__device__ bool solve_adjoint3(const double J[3][3], const double b[3], double x[3]) {
  double M[3][3];
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) M[r][c] = (r == c ? 1.0 : 0.0) - J[c][r];
  const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                     M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                     M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
  if (!(fabs(det) > 0.0) || !isfinite(det)) return false;
  for (int k = 0; k < 3; k++) {
    double A[3][3];
    for (int r = 0; r < 3; r++)
      for (int c = 0; c < 3; c++) A[r][c] = c == k ? b[r] : M[r][c];
    x[k] = (A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
            A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
            A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0])) /
           det;
  }
  return true;
}

// The particle's push constants and start (as map_block sets them up)
template <int D>
__device__ __forceinline__ void vjp_particle(const PView<double> &pv, int64_t i,
                                             const KConst<double> &kc, const MapScale<double> &ms,
                                             PushConst<double> &pc, int cell[3], double off[3],
                                             double dtdx[3]) {
  const int64_t cap = pv.cap;
  const int s_id = pv.sp[i];
  pc.q = pv.w[i] * kc.qs[s_id];
  pc.m = pv.w[i] * kc.ms[s_id];
  pc.inv_m = 1.0 / pc.m;
  pc.mk = pc.m * kc.kappa;
  pc.inv_mk = pc.inv_m / kc.kappa;
  pc.hq = 0.5 * pc.q * kc.dt;
  pc.a_hc = pc.hq * pc.inv_m;
  for (int l = 0; l < 3; l++) {
    cell[l] = l < D ? pv.cell[l * cap + i] : 0;
    off[l] = l < D ? pv.off[l * cap + i] : 0.0;
    dtdx[l] = l < D ? kc.dt * ms.inv_dx[l] : 0.0;
  }
  for (int c = 0; c < 3; c++) {
    pc.Pn[c] = pv.P[c * cap + i];
    pc.Am[c] = pv.Am[c * cap + i];
    pc.pn[c] = pc.Pn[c] - pc.q * pc.Am[c];
  }
  pc.gamma_n = sqrt(1.0 + (pc.pn[0] * pc.pn[0] + pc.pn[1] * pc.pn[1] + pc.pn[2] * pc.pn[2]) *
                              pc.inv_mk * pc.inv_mk);
}

__device__ __forceinline__ PushConst<Dual> dual_push_const(const PushConst<double> &pc) {
  PushConst<Dual> pd;
  pd.q = pc.q; pd.m = pc.m; pd.inv_m = pc.inv_m; pd.mk = pc.mk; pd.inv_mk = pc.inv_mk;
  pd.hq = pc.hq; pd.a_hc = pc.a_hc; pd.gamma_n = pc.gamma_n;
  for (int c = 0; c < 3; c++) {
    pd.Pn[c] = pc.Pn[c];
    pd.Am[c] = pc.Am[c];
    pd.pn[c] = pc.pn[c];
  }
  return pd;
}

__global__ void k_zip_rec(const double *__restrict__ a, Dual *__restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = Dual(a[i]);
}


}  // namespace
