// regularity.cu -- pic_knot_jumps(): the knot-jump regularity diagnostic of
// Sec. 5.3, which separates the C^0 derivatives of degree-one shapes from
// the C^1 ones of quadratic shapes.  A knot is where the B-spline changes
// polynomial piece: the nodes for r = 1, the cell midpoints for r = 2.  At
// every knot along every active axis the field interpolants
// F_h = sum_g F_g S_r(x - x_g) are evaluated at +-eps node units along the
// axis.  The other coordinates sit half a cell from their own knots (on
// the node for r = 2, at the cell centre for r = 1), where the interpolant
// is smooth in them.  The two-sided differences of
// E_shape = -grad phi_h - U_h (Euclidean norm) and of grad A_h (Frobenius
// norm) are maximised over all probes.  One thread per probe (axis, node);
// the maxima by integer atomicMax on the bit patterns of the non-negative
// norms.
#include "map_device.cuh"
#include "trace.cuh"

#include <cmath>
#include <cstring>

namespace {

// The interpolants at the point whose per-dimension stencil centre is node
// c[l] with offset t[l] (node units), for shape degree `order`: E_shape and
// grad A_h (columns per active dimension, physical units).
template <int D>
__device__ void shape_fields(const PGeom &pg, const int c[3], const double t[3], int order,
                             const double *__restrict__ phi, const double *__restrict__ U,
                             const double *__restrict__ A, double E[3], double G[3][3]) {
  double S[3][3], dS[3][3];
  for (int l = 0; l < 3; l++)
    for (int o = 0; o < 3; o++) {
      S[l][o] = o == 1 ? 1.0 : 0.0;  // ignorable dimensions: the node itself
      dS[l][o] = 0.0;
    }
  for (int l = 0; l < D; l++) {
    if (order == 1) lspline<double>(t[l], t[l] >= 0.0, S[l], dS[l]);
    else qspline<double>(t[l], S[l], dS[l]);
  }
  const int base[3] = {0, 0, 0};
  const NodeRows<D> nr(pg, c, base);
  const size_t Ng = (size_t)pg.Ng;
  double gphi[3] = {0.0, 0.0, 0.0}, Uh[3] = {0.0, 0.0, 0.0};
  for (int cc = 0; cc < 3; cc++)
    for (int l = 0; l < 3; l++) G[cc][l] = 0.0;
  for (int oz = 0; oz < (D > 2 ? 3 : 1); oz++)
    for (int oy = 0; oy < (D > 1 ? 3 : 1); oy++)
      for (int ox = 0; ox < 3; ox++) {
        const int g = nr.at(ox, oy, oz);
        const int o[3] = {ox, D > 1 ? oy : 1, D > 2 ? oz : 1};
        const double W = S[0][o[0]] * S[1][o[1]] * S[2][o[2]];
        for (int cc = 0; cc < 3; cc++) Uh[cc] += W * U[cc * Ng + g];
        for (int l = 0; l < D; l++) {
          double Wd = dS[l][o[l]] * pg.inv_dx[l];
          for (int m = 0; m < D; m++)
            if (m != l) Wd *= S[m][o[m]];
          gphi[l] += Wd * phi[g];
          for (int cc = 0; cc < 3; cc++) G[cc][l] += Wd * A[cc * Ng + g];
        }
      }
  for (int cc = 0; cc < 3; cc++) E[cc] = -(cc < D ? gphi[cc] : 0.0) - Uh[cc];
}

template <int D>
__global__ void k_knot_jumps(PGeom pg, int order, double eps, const double *__restrict__ phi,
                             const double *__restrict__ U, const double *__restrict__ A,
                             unsigned long long *__restrict__ out) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)D * pg.Ng) return;
  const int a = (int)(tid / pg.Ng);
  int g = (int)(tid % pg.Ng);
  int node[3] = {0, 0, 0};
  node[0] = g & pg.mask[0];
  if (D > 1) node[1] = (g / pg.n0) & pg.mask[1];
  if (D > 2) node[2] = g / pg.n01;
  double E[2][3], G[2][3][3];
  for (int side = 0; side < 2; side++) {
    int c[3] = {node[0], node[1], node[2]};
    double t[3] = {0.0, 0.0, 0.0};
    for (int l = 0; l < D; l++) {
      if (l != a) {
        // half a cell from the transverse knots: the node (r = 2), the cell
        // centre (r = 1: stencil centre j, offset +1/2)
        t[l] = order == 1 ? 0.5 : 0.0;
      } else if (order == 1) {
        t[l] = side ? eps : -eps;  // the knot is the node itself
      } else if (side) {
        c[l] = node[l] + 1;  // past the midpoint the nearest node is the next one
        t[l] = -0.5 + eps;
      } else {
        t[l] = 0.5 - eps;
      }
    }
    shape_fields<D>(pg, c, t, order, phi, U, A, E[side], G[side]);
  }
  double e2 = 0.0, g2 = 0.0;
  for (int cc = 0; cc < 3; cc++) {
    e2 += (E[1][cc] - E[0][cc]) * (E[1][cc] - E[0][cc]);
    for (int l = 0; l < D; l++) g2 += (G[1][cc][l] - G[0][cc][l]) * (G[1][cc][l] - G[0][cc][l]);
  }
  // non-negative doubles order as their bit patterns
  atomicMax(out, (unsigned long long)__double_as_longlong(sqrt(e2)));
  atomicMax(out + 1, (unsigned long long)__double_as_longlong(sqrt(g2)));
}

}  // namespace

extern "C" int pic_knot_jumps(pic_ctx *ctx, double eps, double *E_jump, double *G_jump) {
  if (!ctx || !E_jump || !G_jump) return PIC_EARG;
  if (!(eps > 0.0) || !(eps < 0.25)) {
    ctx->err = "pic_knot_jumps: eps must lie in (0, 1/4) node units";
    return PIC_EARG;
  }
  if (!ctx->started) {
    ctx->err = "pic_knot_jumps before pic_start";
    return PIC_ESTATE;
  }
  TraceRange trace("pic_knot_jumps");
  const int d = ctx->g.dim, Ng = ctx->g.Ng;
  int e;
  // phi and U in real space (as pic_get_potentials returns them) into scr_r
  CK(cudaMemcpyAsync(ctx->work_h, ctx->phi_h, sizeof(double2) * Ng, cudaMemcpyDeviceToDevice,
                     ctx->st));
  CK(cudaMemcpyAsync(ctx->work_h + Ng, ctx->U_h, sizeof(double2) * 3 * Ng,
                     cudaMemcpyDeviceToDevice, ctx->st));
  if ((e = fft_nd(ctx, ctx->work_h, 4, +1))) return e;
  if ((e = field_complex_to_real(ctx, ctx->work_h, ctx->scr_r, 4, 1.0 / Ng))) return e;
  unsigned long long *res = nullptr;
  CK(cudaMalloc(&res, 2 * sizeof(unsigned long long)));
  struct Free {
    void *p;
    ~Free() { cudaFree(p); }
  } fr{res};
  CK(cudaMemsetAsync(res, 0, 2 * sizeof(unsigned long long), ctx->st));
  const PGeom pg = pgeom(ctx);
  const int64_t nth = (int64_t)d * Ng;
  const unsigned nb = (unsigned)((nth + 255) / 256);
  const double *phi = ctx->scr_r, *U = ctx->scr_r + Ng;
  const int order = ctx->opt.order;
  if (d == 1) k_knot_jumps<1><<<nb, 256, 0, ctx->st>>>(pg, order, eps, phi, U, ctx->A_real, res);
  else if (d == 2) k_knot_jumps<2><<<nb, 256, 0, ctx->st>>>(pg, order, eps, phi, U, ctx->A_real, res);
  else k_knot_jumps<3><<<nb, 256, 0, ctx->st>>>(pg, order, eps, phi, U, ctx->A_real, res);
  KCHECK();
  unsigned long long h[2];
  CK(cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  std::memcpy(E_jump, &h[0], sizeof(double));
  std::memcpy(G_jump, &h[1], sizeof(double));
  return PIC_OK;
}
