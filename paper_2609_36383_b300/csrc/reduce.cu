// reduce.cu -- mesh-vector reductions and updates of the outer current
// iteration (Sec. 4.5, Algorithm 1).
//
//  * resid_sums: r = H - j and, in one pass, the sums behind the RMS norms
//    and the maximum node ratio of Eq. mixed-nonlinear-tests;
//  * dots: the Gram matrix dR^T dR and dR^T r of the type-II Anderson update
//    (Eq. anderson-type-two-update);
//  * axpy_dir / lincomb / diff_into: the update vectors.
// Block partials are summed by a single block in a fixed order, so results
// are identical from run to run.
#include "pic_internal.cuh"

namespace {

constexpr int kT = 256;
constexpr int kMaxBlocks = 1024;

__global__ void k_resid(const double *__restrict__ H, const double *__restrict__ j,
                        double *__restrict__ r, int Ng, double tau_r, double tau_a,
                        double *parts) {
  __shared__ double sh[4][kT / 32];
  double s_r = 0, s_h = 0, s_j = 0, mx = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < Ng; g += gridDim.x * blockDim.x) {
    double rr = 0, hh = 0, jj = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      double hv = H[(size_t)c * Ng + g], jv = j[(size_t)c * Ng + g];
      double rv = hv - jv;
      r[(size_t)c * Ng + g] = rv;
      rr += rv * rv;
      hh += hv * hv;
      jj += jv * jv;
    }
    s_r += rr;
    s_h += hh;
    s_j += jj;
    mx = fmax(mx, sqrt(rr) / (tau_a + 0.5 * tau_r * (sqrt(hh) + sqrt(jj))));
  }
  double v[4] = {s_r, s_h, s_j, mx};
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 4; q++) {
    double x = v[q];
    for (int o = 16; o > 0; o >>= 1) {
      double y = __shfl_down_sync(0xffffffffu, x, o);
      x = (q == 3) ? fmax(x, y) : x + y;
    }
    if (lane == 0) sh[q][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0;
    for (int w = 0; w < kT / 32; w++)
      s = (threadIdx.x == 3) ? fmax(s, sh[threadIdx.x][w]) : s + sh[threadIdx.x][w];
    parts[blockIdx.x * 4 + threadIdx.x] = s;
  }
}

__global__ void k_resid_final(const double *parts, int nb, double *out) {
  __shared__ double sh[4][kT];
  for (int q = 0; q < 4; q++) {
    double s = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
      s = (q == 3) ? fmax(s, parts[b * 4 + q]) : s + parts[b * 4 + q];
    sh[q][threadIdx.x] = s;
  }
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int q = 0; q < 4; q++)
        sh[q][threadIdx.x] = (q == 3) ? fmax(sh[q][threadIdx.x], sh[q][threadIdx.x + st])
                                      : sh[q][threadIdx.x] + sh[q][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = sh[threadIdx.x][0];
}

constexpr int kMaxDots = 48;  // M(M+1)/2 + M for the largest history M = 8

struct DotArgs {
  const double *a[kMaxDots];
  const double *b[kMaxDots];
  int np;
};

__global__ void k_dots(DotArgs da, size_t N, double *parts) {
  __shared__ double sh[kT / 32];
  for (int p = 0; p < da.np; p++) {
    double s = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x)
      s += da.a[p][i] * da.b[p][i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int w = 0; w < kT / 32; w++) t += sh[w];
      parts[(size_t)blockIdx.x * da.np + p] = t;
    }
    __syncthreads();
  }
}

__global__ void k_dots_final(const double *parts, int nb, int np, double *out) {
  __shared__ double sh[kT];
  for (int p = 0; p < np; p++) {
    double s = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += parts[(size_t)b * np + p];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[p] = sh[0];
    __syncthreads();
  }
}

struct Gam {
  double g[PIC_MAX_ANDERSON];
  const double *dJ[PIC_MAX_ANDERSON];
  const double *dR[PIC_MAX_ANDERSON];
};

// dir = beta r - sum_c (dJ_c + beta dR_c) gamma_c
__global__ void k_axpy_dir(double *dir, const double *r, double beta, Gam gm, int mh, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    double s = beta * r[i];
    for (int c = 0; c < mh; c++) s -= (gm.dJ[c][i] + beta * gm.dR[c][i]) * gm.g[c];
    dir[i] = s;
  }
}

__global__ void k_lincomb(double *out, const double *a, double al, const double *b, double be,
                          size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = al * a[i] + be * b[i];
}

__global__ void k_diff(double *out, const double *a, const double *b, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

int grid_for(size_t n) {
  size_t b = (n + kT - 1) / kT;
  if (b > kMaxBlocks) b = kMaxBlocks;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

int resid_launch(pic_ctx *ctx, const double *Hv, const double *jv, double *rv, double tau_r,
                 double tau_a) {
  int Ng = ctx->g.Ng;
  int nb = grid_for(Ng);
  k_resid<<<nb, kT, 0, ctx->st>>>(Hv, jv, rv, Ng, tau_r, tau_a, ctx->red);
  KCHECK();
  k_resid_final<<<1, kT, 0, ctx->st>>>(ctx->red, nb, ctx->red + (size_t)nb * 4);
  KCHECK();
  CK(cudaMemcpyAsync(ctx->red_host, ctx->red + (size_t)nb * 4, sizeof(double) * 4,
                     cudaMemcpyDeviceToHost, ctx->st));
  return PIC_OK;
}

void resid_finish(pic_ctx *ctx, ResidSums *out) {
  out->r2 = ctx->red_host[0];
  out->H2 = ctx->red_host[1];
  out->j2 = ctx->red_host[2];
  out->smax = ctx->red_host[3];
}

int dots(pic_ctx *ctx, const double *const *a, const double *const *b, int npairs, double *out) {
  if (npairs > kMaxDots) {
    ctx->err = "dots: too many pairs";
    return PIC_EARG;
  }
  DotArgs da;
  for (int p = 0; p < npairs; p++) {
    da.a[p] = a[p];
    da.b[p] = b[p];
  }
  da.np = npairs;
  size_t N = (size_t)3 * ctx->g.Ng;
  int nb = grid_for(N);
  k_dots<<<nb, kT, 0, ctx->st>>>(da, N, ctx->red);
  KCHECK();
  k_dots_final<<<1, kT, 0, ctx->st>>>(ctx->red, nb, npairs, ctx->red + (size_t)nb * npairs);
  KCHECK();
  CK(cudaMemcpyAsync(ctx->red_host, ctx->red + (size_t)nb * npairs, sizeof(double) * npairs,
                     cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int p = 0; p < npairs; p++) out[p] = ctx->red_host[p];
  return PIC_OK;
}

int axpy_dir(pic_ctx *ctx, double *dir, const double *r, double beta,
             const double *const *dJ, const double *const *dR, const double *gam, int mh,
             size_t N3) {
  Gam gm;
  for (int c = 0; c < PIC_MAX_ANDERSON; c++) {
    gm.g[c] = c < mh ? gam[c] : 0.0;
    gm.dJ[c] = c < mh ? dJ[c] : nullptr;
    gm.dR[c] = c < mh ? dR[c] : nullptr;
  }
  k_axpy_dir<<<grid_for(N3), kT, 0, ctx->st>>>(dir, r, beta, gm, mh, N3);
  KCHECK();
  return PIC_OK;
}

int lincomb(pic_ctx *ctx, double *out, const double *a, double alpha, const double *b,
            double beta_c, size_t N) {
  k_lincomb<<<grid_for(N), kT, 0, ctx->st>>>(out, a, alpha, b, beta_c, N);
  KCHECK();
  return PIC_OK;
}

int diff_into(pic_ctx *ctx, double *out, const double *a, const double *b, size_t N) {
  k_diff<<<grid_for(N), kT, 0, ctx->st>>>(out, a, b, N);
  KCHECK();
  return PIC_OK;
}
