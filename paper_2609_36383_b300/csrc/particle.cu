// particle.cu -- particle kernels of one simulation context: the launcher of
// the particle map (map_device.cuh), loading and export, step start, commit,
// kinetic energy, point deposits for pic_start, and the counting sort.
#include "map_device.cuh"
#include "csum.cuh"

#include <cmath>
#include <type_traits>

namespace {

// second level of the particle sums (k_psum_level2)
constexpr int kPsumBlocks = 128, kPsumThreads = 256;

// ---- simple per-particle kernels -------------------------------------------
// Loads particles.  Positions come either as absolute coordinates x (cin
// null), from which the nearest node and the offset are formed, or directly
// in the stored form (cin: nearest node per dimension in [0, n), x: the
// offset in node units in [-1/2, 1/2)); a stored-form entry out of range is
// replaced by node 0, offset 0 and reported through *bad (bit 2).
template <int D, typename T>
__global__ void k_load(int64_t n, int64_t cap, const double *__restrict__ x,
                       const int32_t *__restrict__ cin, const double *__restrict__ uP,
                       int canonical, const double *__restrict__ w,
                       const int32_t *__restrict__ sp, int nspecies, PGeom pg, int32_t *cell,
                       T *off, T *P, double *u_in, double *wo, int32_t *spo, int64_t *id,
                       unsigned int *bad) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int l = 0; l < D; l++) {
    int c;
    double o;
    if (cin) {
      c = cin[l * n + i];
      o = x[l * n + i];
      if (c < 0 || c >= pg.n[l] || !(o >= -0.5 && o < 0.5)) {
        atomicOr(bad, 2u);
        c = 0;
        o = 0.0;
      }
    } else {
      double u = (x[l * n + i] - pg.x0[l]) * pg.inv_dx[l];
      double nn = (double)pg.n[l];
      u -= nn * floor(u / nn);
      c = (int)floor(u + 0.5);
      o = u - (double)c;
      if (c >= pg.n[l]) c -= pg.n[l];
    }
    cell[l * cap + i] = c;
    off[l * cap + i] = (T)o;
  }
  for (int c = 0; c < 3; c++) {
    if (canonical) P[c * cap + i] = (T)uP[c * n + i];
    else u_in[c * cap + i] = uP[c * n + i];
  }
  wo[i] = w[i];
  // a species index outside [0, nspecies) is stored as 0, so that no kernel
  // indexes the species tables with it, and reported through *bad
  int s = sp ? sp[i] : 0;
  if (s < 0 || s >= nspecies) {
    atomicOr(bad, 1u);
    s = 0;
  }
  spo[i] = s;
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
  for (int l = 0; l < D; l++) spline_val<double>(pg.order, off[l], Sw[l]);
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

// step start (Algorithm 1, first line): A^- = A^n_h(x^n), p^n = P^n - q A^-, v^0 = v(p^n),
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
// (Eq. Kkin-nondim): per particle in the particle real type, summed in FP64:
// plainly within a warp, with compensation across warps and blocks (block
// (sum, error) pairs merged on the host)
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
  // a warp's 32 positive terms summed plainly (a 5-level tree: a few ulps of
  // the warp's sum, errors independent from warp to warp, and 5 FP64 adds a
  // lane instead of 5 TwoSums); warps and blocks merged with compensation
  double kw = widen(k);
  for (int o = 16; o > 0; o >>= 1) kw += __shfl_down_sync(0xffffffffu, kw, o);
  __shared__ double sh[kPT / 32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = kw;
  __syncthreads();
  if (threadIdx.x == 0) {
    CSum t = csum_zero();
    for (int w = 0; w < kPT / 32; w++) csum_add(t, sh[w]);
    psum[2 * blockIdx.x] = t.s;
    psum[2 * blockIdx.x + 1] = t.c;
  }
}

// Second level of the particle sums, on the device: the nb block partials
// at in[2b], in[2b + 1] (two plain quantities, pairs = 0, or one (sum,
// error) pair, pairs = 1) merged with compensation by kPsumBlocks blocks,
// each over a contiguous range, into out[4k .. 4k + 3] = (sum, error) of
// the first and of the second quantity.  Fixed order, so reproducible; the
// host then merges kPsumBlocks entries instead of nb.
__global__ void __launch_bounds__(kPsumThreads)
k_psum_level2(const double *__restrict__ in, int64_t nb, int pairs, double *__restrict__ out) {
  const int64_t lo = nb * blockIdx.x / kPsumBlocks, hi = nb * (blockIdx.x + 1) / kPsumBlocks;
  CSum a = csum_zero(), b = csum_zero();
  for (int64_t i = lo + threadIdx.x; i < hi; i += kPsumThreads) {
    if (pairs) {
      a = csum_merge(a, CSum{in[2 * i], in[2 * i + 1]});
    } else {
      csum_add(a, in[2 * i]);
      csum_add(b, in[2 * i + 1]);
    }
  }
  a = csum_warp(a);
  b = csum_warp(b);
  __shared__ CSum sa[kPsumThreads / 32], sb[kPsumThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = a;
    sb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    CSum ta = csum_zero(), tb = csum_zero();
    for (int w = 0; w < kPsumThreads / 32; w++) {
      ta = csum_merge(ta, sa[w]);
      tb = csum_merge(tb, sb[w]);
    }
    out[4 * blockIdx.x] = ta.s;
    out[4 * blockIdx.x + 1] = ta.c;
    out[4 * blockIdx.x + 2] = tb.s;
    out[4 * blockIdx.x + 3] = tb.c;
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

// u = (P - q A_h(x)) / m in load order
template <int D, typename T>
__global__ void k_export_u(PView<T> pv, const int64_t *__restrict__ id, const double *__restrict__ A,
                           PGeom pg, KConst<T> kc, double *u) {
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
  double q = pv.w[i] * kc.qs[s], m = pv.w[i] * kc.ms[s];
  int64_t j = id[i], n = pv.np;
  for (int c = 0; c < 3; c++) u[c * n + j] = ((double)pv.P[c * pv.cap + i] - q * Ax[c]) / m;
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
  v.drec = ctx->dep_rec;
  return v;
}

StepConst base_sc(const pic_ctx *ctx) {
  StepConst sc;
  memset(&sc, 0, sizeof sc);
  sc.dt = ctx->dt;
  sc.kappa = ctx->opt.kappa;
  sc.order = ctx->opt.order;
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
                   (void **)&ctx->tmp_l, (void **)&ctx->dep_rec};
  for (void **b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  // a whole number of map chunks, so that the map's staging copies of a
  // chunk stay inside every array and start on 16-byte boundaries
  int64_t cap = ((n > 0 ? n : 1) + kChunkMax - 1) / kChunkMax * kChunkMax;
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
  if (R == 4) CK(cudaMalloc((void **)&ctx->dep_rec, 2 * sizeof(float4) * cap));
  CK(cudaMalloc((void **)&ctx->u_in, sizeof(double) * 3 * cap));
  CK(cudaMalloc((void **)&ctx->tmp_d, sizeof(double) * 7 * cap));
  CK(cudaMalloc((void **)&ctx->tmp_i, sizeof(int32_t) * 4 * cap));
  CK(cudaMalloc((void **)&ctx->keys, sizeof(int32_t) * cap));
  CK(cudaMalloc((void **)&ctx->tmp_l, sizeof(int64_t) * cap));
  CK(cudaMalloc((void **)&ctx->psum, sizeof(double) * (4 * nb + 4 * kPsumBlocks) + 64));
  if (ctx->psum_host) cudaFreeHost(ctx->psum_host);
  ctx->psum_host = nullptr;
  CK(cudaMallocHost((void **)&ctx->psum_host, sizeof(double) * (4 * nb + 4 * kPsumBlocks) + 64));
  CK(cudaMemsetAsync(ctx->cell, 0, sizeof(int32_t) * 3 * cap, ctx->st));
  CK(cudaMemsetAsync(ctx->off, 0, R * 3 * cap, ctx->st));
  ctx->cap = cap;
  return PIC_OK;
}

int particles_load(pic_ctx *ctx, const int32_t *sp, const int32_t *cell_in, const double *x,
                   const double *uP, int canonical, const double *w, int on_device) {
  int64_t n = ctx->np, cap = ctx->cap;
  if (n == 0) return PIC_OK;
  const int d = ctx->g.dim;
  const double *dx = x, *du = uP, *dw = w;
  const int32_t *dsp = sp, *dcell = cell_in;
  if (cell_in && !on_device) {  // staged after the species staging area
    CK(cudaMemcpyAsync(ctx->tmp_i + cap, cell_in, sizeof(int32_t) * d * n,
                       cudaMemcpyHostToDevice, ctx->st));
    dcell = ctx->tmp_i + cap;
  }
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
  CK(cudaMemsetAsync(ctx->cnt_dev, 0, sizeof(EvalCounters), ctx->st));
  PIC_DISPATCH(ctx, (k_load<DD, RT><<<nblk(n), kPT, 0, ctx->st>>>(
                         n, cap, dx, dcell, du, canonical, dw, dsp,
                         ctx->nspecies, pg, ctx->cell, (RT *)ctx->off, (RT *)ctx->P, ctx->u_in,
                         ctx->w, ctx->sp, ctx->id, &ctx->cnt_dev->status)));
  KCHECK();
  CK(cudaMemcpyAsync(ctx->cnt_host, ctx->cnt_dev, sizeof(EvalCounters), cudaMemcpyDeviceToHost,
                     ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (ctx->cnt_host->status) {
    ctx->err = ctx->cnt_host->status & 1u ? "pic_set_particles: species index out of range"
                                          : "pic_set_particles: node index or offset out of range";
    return PIC_EARG;
  }
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

// The common path's particle map: the inner-solve launch, then the deposit
// launch, over chunks of kChunkOf<RT> particles.
template <int DD, typename RT, bool FIN>
int map_split_launch(pic_ctx *ctx, int nb, int nr, const PGeom &pg, const StepConst &sc,
                     unsigned long long *tim) {
  const KConst<RT> kc = kconst<RT>(sc, pg);
  if constexpr (std::is_same<RT, double>::value) {
    // FP64: one persistent launch (k_map_fused), as many CTAs as fit at once
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_map_fused<DD, RT, FIN>, kPT, 0));
    int grid = (per_sm > 0 ? per_sm : 1) * ctx->num_sms;
    grid = grid < nb ? grid : nb;
    k_map_fused<DD, RT, FIN><<<grid, kPT, 0, ctx->st>>>(pview<RT>(ctx), (const RT *)ctx->nodes,
                                                        (const RT *)ctx->nodes_u, ctx->Jorb, pg,
                                                        kc, ctx->cnt_dev, ctx->psum, tim, nb, nr);
    return PIC_OK;
  }
  // FP32: the chunk's inputs staged in dynamic shared memory
  const int dsm = kStaged<RT, RT> ? Stage<DD, RT>::kBytes : 0;
  if (dsm)
    CK(cudaFuncSetAttribute(k_map_solve<DD, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            dsm));
  k_map_solve<DD, RT><<<nb, kPT, dsm, ctx->st>>>(pview<RT>(ctx), (const RT *)ctx->nodes, pg, kc,
                                                 ctx->cnt_dev, tim, nr);
  k_map_deposit<DD, RT, FIN><<<nb, kPT, 0, ctx->st>>>(pview<RT>(ctx), (const RT *)ctx->nodes,
                                                      (const RT *)ctx->nodes_u, ctx->Jorb, pg, kc,
                                                      ctx->cnt_dev, ctx->psum, tim, nr);
  return PIC_OK;
}

// The same for the FP32 stage of an FP64 context: FP32 arithmetic and FP32
// node records on the FP64 particle storage.
template <int DD, bool FIN>
void map_split_launch_f32(pic_ctx *ctx, int nb, int nr, const PGeom &pg, const StepConst &sc,
                          unsigned long long *tim) {
  const KConst<float> kc = kconst<float>(sc, pg);
  k_map_solve<DD, float, double><<<nb, kPT, 0, ctx->st>>>(pview<double>(ctx), ctx->nodes_f, pg,
                                                          kc, ctx->cnt_dev, tim, nr);
  k_map_deposit<DD, float, FIN, double><<<nb, kPT, 0, ctx->st>>>(
      pview<double>(ctx), ctx->nodes_f, ctx->nodes_u_f, ctx->Jorb, pg, kc, ctx->cnt_dev,
      ctx->psum, tim, nr);
}

// Groups of kPT particles per chunk of the common-path map: as many as keep
// at least two chunks per resident CTA slot (slots = CTAs per SM x SMs), at
// most maxr, at least one, and a power of two: the chunk then divides the
// capacity granule kChunkMax, so a chunk's staging copies never read past
// the particle arrays.  Long chunks shorten the share of each chunk's drain;
// short ones keep every SM busy on small problems.
int chunk_groups(int64_t np, int maxr, int64_t slots) {
  const int64_t r = np / ((int64_t)kPT * 2 * (slots > 0 ? slots : 1));
  int g = 1;
  while (2 * g <= maxr && 2 * g <= r) g *= 2;
  return g;
}

int particles_map_launch(pic_ctx *ctx, const StepConst &sc_in, int final_pass) {
  CK(cudaMemsetAsync(ctx->cnt_dev, 0, sizeof(EvalCounters), ctx->st));
  int nb = nblk(ctx->np);
  ctx->map_final = final_pass;
  // in the device-controlled step's graphs the map kernel times itself and
  // the controller reads its counters on the device
  const bool loop = ctx->loop_capture != 0;
  if (ctx->np > 0) {
    PGeom pg = pgeom(ctx);
    // inside a stream capture the records must become event nodes of the graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(ctx->st, &cap));
    const unsigned evf = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    if (!loop) CK(cudaEventRecordWithFlags(ctx->ev0, ctx->st, evf));
    unsigned long long *tim = loop ? ctx->map_timer : nullptr;
    // the common path runs the lane-refill map over chunks of kChunkOf<RT>
    // particles; the general path one particle per thread
    int nr = 1;
    if (!(sc_in.order != 2 || sc_in.refine_max > 0)) {
      // resident CTAs per SM of the chunk kernels: 2 for FP64 (254
      // registers), 4 for FP32 (128 registers)
      const bool f64 = ctx->rsize == 8 && !ctx->eval_f32;
      nr = chunk_groups(ctx->np, f64 ? kRefillOf<double> : kRefillOf<float>,
                        (int64_t)(f64 ? 2 : 4) * ctx->num_sms);
      nb = (int)((ctx->np + nr * kPT - 1) / (nr * kPT));
    }
#define PIC_MAP_LAUNCH(FIN, GEN)                                                          \
  PIC_DISPATCH(ctx, (k_map<DD, RT, FIN, GEN><<<nb, kPT, 0, ctx->st>>>(                      \
                         pview<RT>(ctx), (const RT *)ctx->nodes, (const RT *)ctx->nodes_u, \
                         ctx->Jorb, pg, kconst<RT>(sc_in, pg), ctx->cnt_dev, ctx->psum, tim)))
    // the common path: inner solves, then deposits (two launches)
    int e_split = PIC_OK;
#define PIC_MAP_SPLIT(FIN) \
  PIC_DISPATCH(ctx, (e_split = map_split_launch<DD, RT, FIN>(ctx, nb, nr, pg, sc_in, tim)))
    // the general kernels (degree-one shapes, refinement) only when needed
    const bool gen = sc_in.order != 2 || sc_in.refine_max > 0;
    if (ctx->eval_f32) {  // FP32 arithmetic on the FP64 particle storage
#define PIC_MAP_F32(DD, FIN, GEN) map_split_launch_f32<DD, FIN>(ctx, nb, nr, pg, sc_in, tim)
#define PIC_MAP_F32_D(FIN, GEN)                                                            \
  do {                                                                                     \
    if (ctx->g.dim == 1) PIC_MAP_F32(1, FIN, GEN);                                         \
    else if (ctx->g.dim == 2) PIC_MAP_F32(2, FIN, GEN);                                    \
    else PIC_MAP_F32(3, FIN, GEN);                                                         \
  } while (0)
      // the FP32 stage runs plain evaluations of the common path only
      // (pic_init admits fp32_first with quadratic shapes and no refinement)
      if (final_pass || gen) {
        ctx->err = "FP32 stage: final pass or general shapes requested";
        return PIC_EARG;
      }
      PIC_MAP_F32_D(false, false);
#undef PIC_MAP_F32_D
#undef PIC_MAP_F32
    } else if (final_pass) {
      if (gen) PIC_MAP_LAUNCH(true, true);
      else PIC_MAP_SPLIT(true);
    } else {
      if (gen) PIC_MAP_LAUNCH(false, true);
      else PIC_MAP_SPLIT(false);
    }
#undef PIC_MAP_SPLIT
#undef PIC_MAP_LAUNCH
    if (e_split) return e_split;
    KCHECK();
    if (!loop) CK(cudaEventRecordWithFlags(ctx->ev1, ctx->st, evf));
    if (ctx->opt.deterministic_deposit) {  // replaces the atomic deposit in Jorb
      int e = det_deposit(ctx, ctx->Jorb, sc_in);
      if (e) return e;
    }
    if (final_pass) {  // the work and chain-rule sums: block partials merged on the device
      k_psum_level2<<<kPsumBlocks, kPsumThreads, 0, ctx->st>>>(ctx->psum, nb, 0,
                                                              ctx->psum + 2 * (size_t)nb);
      KCHECK();
      CK(cudaMemcpyAsync(ctx->psum_host, ctx->psum + 2 * (size_t)nb,
                         sizeof(double) * 4 * kPsumBlocks, cudaMemcpyDeviceToHost, ctx->st));
    }
  }
  if (!loop)
    CK(cudaMemcpyAsync(ctx->cnt_host, ctx->cnt_dev, sizeof(EvalCounters),
                       cudaMemcpyDeviceToHost, ctx->st));
  return PIC_OK;
}

void particles_final_sums(const pic_ctx *ctx, double *work, double *chain) {
  // fixed order, compensated: reproducible diagnostics
  const double *ps = ctx->psum_host;  // kPsumBlocks (sum, error) pairs of each
  CSum cw = csum_zero(), cc = csum_zero();
  for (int k = 0; k < kPsumBlocks; k++) {
    cw = csum_merge(cw, CSum{ps[4 * k], ps[4 * k + 1]});
    cc = csum_merge(cc, CSum{ps[4 * k + 2], ps[4 * k + 3]});
  }
  *work = csum_value(cw);
  *chain = csum_value(cc);
}

int particles_map_finish(pic_ctx *ctx, double *work_sum, double *chain_sum, EvalCounters *cnt) {
  double work = 0.0, chain = 0.0;
  if (ctx->np > 0) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    ctx->map_ms += ms;
    ctx->map_launches++;
    if (ctx->map_final) particles_final_sums(ctx, &work, &chain);
  }
  *cnt = *ctx->cnt_host;
  ctx->pushes += ctx->np;
  ctx->inner_iters += (long long)cnt->inner_sum;
  ctx->pieces += (long long)cnt->pieces;
  ctx->refined += (long long)cnt->refined;
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

// The same queued: the kinetic partials are copied to psum_host and merged
// by particles_kinetic_collect after the caller's synchronisation.
int particles_kinetic_queued(pic_ctx *ctx) {
  if (ctx->np == 0) return PIC_OK;
  PGeom pg = pgeom(ctx);
  StepConst sc = base_sc(ctx);
  int nb = nblk(ctx->np);
  PIC_DISPATCH(ctx, (k_kinetic<DD, RT><<<nb, kPT, 0, ctx->st>>>(
                         pview<RT>(ctx), A_typed<RT>(ctx), pg, kconst<RT>(sc, pg), ctx->psum)));
  KCHECK();
  k_psum_level2<<<kPsumBlocks, kPsumThreads, 0, ctx->st>>>(ctx->psum, nb, 1,
                                                          ctx->psum + 2 * (size_t)nb);
  KCHECK();
  CK(cudaMemcpyAsync(ctx->psum_host, ctx->psum + 2 * (size_t)nb,
                     sizeof(double) * 4 * kPsumBlocks, cudaMemcpyDeviceToHost, ctx->st));
  return PIC_OK;
}

double particles_kinetic_collect(const pic_ctx *ctx) {
  if (ctx->np == 0) return 0.0;
  const double *ps = ctx->psum_host;
  CSum k = csum_zero();
  for (int b = 0; b < kPsumBlocks; b++) k = csum_merge(k, CSum{ps[4 * b], ps[4 * b + 1]});
  return csum_value(k);
}

int particles_kinetic(pic_ctx *ctx, double *K) {
  if (ctx->np == 0) { *K = 0.0; return PIC_OK; }
  PGeom pg = pgeom(ctx);
  StepConst sc = base_sc(ctx);
  int nb = nblk(ctx->np);
  PIC_DISPATCH(ctx, (k_kinetic<DD, RT><<<nb, kPT, 0, ctx->st>>>(
                         pview<RT>(ctx), A_typed<RT>(ctx), pg, kconst<RT>(sc, pg), ctx->psum)));
  KCHECK();
  k_psum_level2<<<kPsumBlocks, kPsumThreads, 0, ctx->st>>>(ctx->psum, nb, 1,
                                                          ctx->psum + 2 * (size_t)nb);
  KCHECK();
  CK(cudaMemcpyAsync(ctx->psum_host, ctx->psum + 2 * (size_t)nb,
                     sizeof(double) * 4 * kPsumBlocks, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  const double *ps = ctx->psum_host;
  CSum k = csum_zero();
  for (int b = 0; b < kPsumBlocks; b++) k = csum_merge(k, CSum{ps[4 * b], ps[4 * b + 1]});
  *K = csum_value(k);
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

int particles_export_u(pic_ctx *ctx, double *u, int on_device) {
  int64_t n = ctx->np;
  if (n == 0) return PIC_OK;
  double *du = on_device ? u : ctx->tmp_d;
  PGeom pg = pgeom(ctx);
  StepConst sc = base_sc(ctx);
  PIC_DISPATCH(ctx, (k_export_u<DD, RT><<<nblk(n), kPT, 0, ctx->st>>>(
                         pview<RT>(ctx), ctx->id, ctx->A_real, pg, kconst<RT>(sc, pg), du)));
  KCHECK();
  if (!on_device)
    CK(cudaMemcpyAsync(u, du, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->st));
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

// ---- counting sort of the particles by cell ------------------------------
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
  int e;
  if (ctx->opt.deterministic_deposit && ctx->det_count) {
    // the same cell order, with the order inside a cell fixed
    if ((e = det_sort_slots(ctx, ctx->tmp_l))) return e;
  } else {
    CK(cudaMemsetAsync(ctx->cnt_sort, 0, sizeof(int32_t) * g.Ng, ctx->st));
    k_sort_keys<<<nblk(ctx->np), kPT, 0, ctx->st>>>(ctx->np, ctx->cap, ctx->cell, g.dim, g.n[0],
                                                    g.n[0] * g.n[1], ctx->keys, ctx->cnt_sort);
    KCHECK();
    k_sort_scan<<<1, 1024, 0, ctx->st>>>(ctx->cnt_sort, g.Ng);
    KCHECK();
    k_sort_slots<<<nblk(ctx->np), kPT, 0, ctx->st>>>(ctx->np, ctx->keys, ctx->cnt_sort,
                                                     ctx->tmp_l);
    KCHECK();
  }
  if ((e = permute_field<int32_t>(ctx, ctx->cell, g.dim))) return e;
  if (ctx->rsize == 8) {
    if ((e = permute_field<double>(ctx, (double *)ctx->off, g.dim))) return e;
    if ((e = permute_field<double>(ctx, (double *)ctx->P, 3))) return e;
  } else {
    if ((e = permute_field<float>(ctx, (float *)ctx->off, g.dim))) return e;
    if ((e = permute_field<float>(ctx, (float *)ctx->P, 3))) return e;
  }
  if (ctx->tan) {  // the forward sensitivity travels with its particles
    if ((e = permute_field<double>(ctx, ctx->tan->off, g.dim))) return e;
    if ((e = permute_field<double>(ctx, ctx->tan->P, 3))) return e;
  }
  if ((e = permute_field<double>(ctx, ctx->w, 1))) return e;
  if ((e = permute_field<int32_t>(ctx, ctx->sp, 1))) return e;
  if ((e = permute_field<int64_t>(ctx, ctx->id, 1))) return e;
  CK(cudaStreamSynchronize(ctx->st));
  return PIC_OK;
}
