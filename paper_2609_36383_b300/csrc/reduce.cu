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
#include "csum.cuh"

namespace {

constexpr int kT = 256;
constexpr int kMaxBlocks = 1024;

// r = H - j; per block the compensated sums of |r|^2, |H|^2, |j|^2 as
// (sum, error) pairs and the largest scaled node residual (8 doubles)
__global__ void k_resid(const double *__restrict__ H, const double *__restrict__ j,
                        double *__restrict__ r, int Ng, double tau_r, double tau_a,
                        double *parts) {
  __shared__ CSum sh[3][kT / 32];
  __shared__ double shm[kT / 32];
  CSum acc[3] = {csum_zero(), csum_zero(), csum_zero()};
  double mx = 0;
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
    csum_add(acc[0], rr);
    csum_add(acc[1], hh);
    csum_add(acc[2], jj);
    mx = fmax(mx, sqrt(rr) / (tau_a + 0.5 * tau_r * (sqrt(hh) + sqrt(jj))));
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 3; q++) {
    CSum x = csum_warp(acc[q]);
    if (lane == 0) sh[q][wid] = x;
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if (lane == 0) shm[wid] = mx;
  __syncthreads();
  if (threadIdx.x < 3) {
    CSum t = csum_zero();
    for (int w = 0; w < kT / 32; w++) t = csum_merge(t, sh[threadIdx.x][w]);
    parts[blockIdx.x * 8 + 2 * threadIdx.x] = t.s;
    parts[blockIdx.x * 8 + 2 * threadIdx.x + 1] = t.c;
  } else if (threadIdx.x == 3) {
    double m = 0;
    for (int w = 0; w < kT / 32; w++) m = fmax(m, shm[w]);
    parts[blockIdx.x * 8 + 6] = m;
  }
}

__global__ void k_resid_final(const double *parts, int nb, double *out) {
  __shared__ CSum sh[3][kT];
  __shared__ double shm[kT];
  for (int q = 0; q < 3; q++) {
    CSum t = csum_zero();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
      t = csum_merge(t, CSum{parts[b * 8 + 2 * q], parts[b * 8 + 2 * q + 1]});
    sh[q][threadIdx.x] = t;
  }
  double m = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = fmax(m, parts[b * 8 + 6]);
  shm[threadIdx.x] = m;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      for (int q = 0; q < 3; q++) sh[q][threadIdx.x] = csum_merge(sh[q][threadIdx.x], sh[q][threadIdx.x + st]);
      shm[threadIdx.x] = fmax(shm[threadIdx.x], shm[threadIdx.x + st]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 3) out[threadIdx.x] = csum_value(sh[threadIdx.x][0]);
  else if (threadIdx.x == 3) out[3] = shm[0];
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
  k_resid_final<<<1, kT, 0, ctx->st>>>(ctx->red, nb, ctx->red + (size_t)nb * 8);
  KCHECK();
  CK(cudaMemcpyAsync(ctx->red_host, ctx->red + (size_t)nb * 8, sizeof(double) * 4,
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
