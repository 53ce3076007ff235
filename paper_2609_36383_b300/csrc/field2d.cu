// field2d.cu -- the spectral field step of one map evaluation on a 2D mesh
// in three launches (Sec. 4.5, current-based formulation; Eq. CN-field).
//
// The generic path transforms, updates and packs in eight launches of small
// kernels (r2c, two forward axis FFTs, the CN mode update, two inverse axis
// FFTs, the record packing, a memset), each a few microseconds long on the
// meshes of this method.  Here the same arithmetic runs as
//   1. k_f2_rows_fwd: the trial current, real, transformed along x by rows;
//   2. k_f2_cols_cn:  per column, the forward transform along y, the
//      Nyquist projection, continuity and the CN update of every mode of the
//      column (writing the candidate n+1 spectra), then the inverse
//      transforms along y of the gather spectra (i k phi^{1/2}, A^{n+1} and,
//      on the final pass, U^{n+1/2}), all in shared memory;
//   3. k_f2_rows_pack: per row, the inverse transforms along x, the node
//      records (grad phi^{1/2}, A^n, A^{n+1}) in the particle real type, the
//      real copy of A^{n+1}, and the cleared deposit target J_orb; on the
//      final pass also the real-space gather fields kept for the mesh side
//      of the work residual.
// The transforms are the radix-2 decimation-in-time butterflies of fft.cu
// (same twiddle tables, same unnormalised convention), so results agree with
// the generic path to rounding.
// On a 1D mesh of at most kF1MaxN nodes the same step is one launch of one
// CTA (k_f1_field): forward transform, CN update, inverse transforms and
// node records, all in shared memory.
#include "pic_internal.cuh"

#include <cmath>

namespace {

// In-place radix-2 DIT FFT of nl lines of N = 2^logN points stored one after
// another in shared memory, each loaded in bit-reversed order.  Unnormalised;
// the inverse conjugates the twiddles.  Ends with a barrier.
__device__ __forceinline__ void fft_lines(double2 *sm, int nl, int logN,
                                          const double2 *__restrict__ tw, bool inverse) {
  const int logHalf = logN - 1;
  const int tot = nl << logHalf;
  for (int lh = 0; lh < logN; lh++) {
    const int h = 1 << lh;
    const int tshift = logN - 1 - lh;  // twiddle stride N / (2h)
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
      const int b = t >> logHalf, j = t & ((1 << logHalf) - 1);
      const int grp = j >> lh, pos = j & (h - 1);
      const int i0 = (b << logN) + (grp << (lh + 1)) + pos, i1 = i0 + h;
      double2 wv = __ldg(tw + (pos << tshift));
      if (inverse) wv.y = -wv.y;
      const double2 x0 = sm[i0], x1 = sm[i1];
      double2 y;
      y.x = wv.x * x1.x - wv.y * x1.y;
      y.y = wv.x * x1.y + wv.y * x1.x;
      sm[i0] = make_double2(x0.x + y.x, x0.y + y.y);
      sm[i1] = make_double2(x0.x - y.x, x0.y - y.y);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int brev_n(int k, int logN) {
  return (int)(__brev((unsigned)k) >> (32 - logN));
}

// 1. rows of the real trial current -> x-transformed spectra (3 components):
// grid (n1 / rpc, 3), rpc rows per CTA
__global__ void k_f2_rows_fwd(const double *__restrict__ jt, double2 *__restrict__ jh, int n0,
                              int log0, int Ng, int rpc, const double2 *__restrict__ tw0) {
  extern __shared__ double2 sm[];
  const int c = blockIdx.y, row0 = blockIdx.x * rpc;
  const double *in = jt + (size_t)c * Ng + (size_t)row0 * n0;
  double2 *out = jh + (size_t)c * Ng + (size_t)row0 * n0;
  const int tot = rpc * n0;
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const int b = t >> log0, x = t & (n0 - 1);
    sm[(b << log0) + brev_n(x, log0)] = make_double2(in[t], 0.0);
  }
  __syncthreads();
  fft_lines(sm, rpc, log0, tw0, false);
  for (int t = threadIdx.x; t < tot; t += blockDim.x) out[t] = sm[t];
}

struct ColArgs {
  const double2 *jh;                                  // x-transformed J (3 comps)
  const double2 *rho, *phi, *psi, *A, *U;             // accepted state spectra
  double2 *rho1, *phi1, *psi1, *A1, *U1;              // candidate n+1 spectra
  double2 *out;                                       // nc gather spectra, y-inverse-transformed
  const double2 *tw1;
  int n0, n1, log1, Ng, dim, nc, project;
  double kx_scale, ky_scale;                          // 2 pi / L per axis
  double dt, kap2, sigma1, sigma2;
};

__device__ __forceinline__ double2 c_i(double s, double2 z) {  // (i s) z
  return make_double2(-s * z.y, s * z.x);
}

// One CN mode update for the pair (f, g) (as field.cu's cn_mode)
__device__ __forceinline__ void cn_pair(double a, double b, double2 f, double2 gg, double2 src,
                                        double2 *f1, double2 *g1) {
  double inv = 1.0 / (1.0 + a * b);
  double c1 = (1.0 - a * b) * inv, c2 = -2.0 * b * inv;
  double2 gn = make_double2((c1 * gg.x + c2 * f.x + src.x * inv),
                            (c1 * gg.y + c2 * f.y + src.y * inv));
  *g1 = gn;
  *f1 = make_double2(f.x + a * (gn.x + gg.x), f.y + a * (gn.y + gg.y));
}

// 2. one column x per CTA: forward y transform of J, CN update of the
// column's modes, inverse y transforms of the gather spectra
__global__ void k_f2_cols_cn(ColArgs p) {
  extern __shared__ double2 sm[];
  const int x = blockIdx.x, n1 = p.n1, Ng = p.Ng, n0 = p.n0;
  double2 *sj = sm;               // 3 lines of n1
  double2 *so = sm + 3 * n1;      // nc lines of n1
  for (int t = threadIdx.x; t < 3 * n1; t += blockDim.x) {
    const int c = t / n1, y = t - c * n1;
    sj[c * n1 + brev_n(y, p.log1)] = p.jh[(size_t)c * Ng + (size_t)y * n0 + x];
  }
  __syncthreads();
  fft_lines(sj, 3, p.log1, p.tw1, false);
  // the mode symbols of this column (zero on a Nyquist index)
  const int ix = x < n0 / 2 ? x : x - n0;
  const bool nyq_x = x == n0 / 2;
  const double kx = nyq_x ? 0.0 : p.kx_scale * ix;
  const double2 z = make_double2(0.0, 0.0);
  const double a = 0.5 * p.dt;
  for (int y = threadIdx.x; y < n1; y += blockDim.x) {
    const size_t g = (size_t)y * n0 + x;
    const int yr = brev_n(y, p.log1);
    const bool nyq_y = y == n1 / 2;
    const int iy = y < n1 / 2 ? y : y - n1;
    const double ky = nyq_y ? 0.0 : p.ky_scale * iy;
    if ((nyq_x || nyq_y) && p.project) {
      p.rho1[g] = z; p.phi1[g] = z; p.psi1[g] = z;
      for (int c = 0; c < 3; c++) { p.A1[c * (size_t)Ng + g] = z; p.U1[c * (size_t)Ng + g] = z; }
      for (int c = 0; c < p.nc; c++) so[c * n1 + yr] = z;
      continue;
    }
    const double k[3] = {kx, ky, 0.0};
    const double k2 = kx * kx + ky * ky;
    const double2 j[3] = {sj[y], sj[n1 + y], sj[2 * n1 + y]};
    // continuity: rho' = rho - dt (i k . j)
    const double2 divj = make_double2(-(k[0] * j[0].y + k[1] * j[1].y + k[2] * j[2].y),
                                      k[0] * j[0].x + k[1] * j[1].x + k[2] * j[2].x);
    const double2 rho0 = p.rho[g];
    const double2 rho1 = make_double2(rho0.x - p.dt * divj.x, rho0.y - p.dt * divj.y);
    const double2 rhoh = make_double2(0.5 * (rho0.x + rho1.x), 0.5 * (rho0.y + rho1.y));
    const double b = 0.5 * p.dt * p.kap2 * k2;
    double2 phi1, psi1;
    const double2 phi0 = p.phi[g];
    const double sr = p.dt * p.kap2 * p.sigma1;
    cn_pair(a, b, phi0, p.psi[g], make_double2(sr * rhoh.x, sr * rhoh.y), &phi1, &psi1);
    p.rho1[g] = rho1; p.phi1[g] = phi1; p.psi1[g] = psi1;
    const double2 phih = make_double2(0.5 * (phi0.x + phi1.x), 0.5 * (phi0.y + phi1.y));
    for (int c = 0; c < p.dim; c++) so[c * n1 + yr] = c_i(k[c], phih);
    const double sj2 = p.dt * p.kap2 * p.sigma2;
    for (int c = 0; c < 3; c++) {
      const double2 A0 = p.A[c * (size_t)Ng + g], U0 = p.U[c * (size_t)Ng + g];
      double2 A1, U1;
      cn_pair(a, b, A0, U0, make_double2(sj2 * j[c].x, sj2 * j[c].y), &A1, &U1);
      p.A1[c * (size_t)Ng + g] = A1;
      p.U1[c * (size_t)Ng + g] = U1;
      so[(p.dim + c) * n1 + yr] = A1;
      if (p.nc > p.dim + 3)
        so[(p.dim + 3 + c) * n1 + yr] = make_double2(0.5 * (U0.x + U1.x), 0.5 * (U0.y + U1.y));
    }
  }
  __syncthreads();
  fft_lines(so, p.nc, p.log1, p.tw1, true);
  for (int t = threadIdx.x; t < p.nc * n1; t += blockDim.x) {
    const int c = t / n1, y = t - c * n1;
    p.out[(size_t)c * Ng + (size_t)y * n0 + x] = so[t];
  }
}

struct RowArgs {
  double2 *spec;             // nc gather spectra (y-inverse-transformed); on the final
                             // pass overwritten with their real-space values (times Ng)
  const double *A_n;         // A^n in real space
  double *A1_real;           // A^{n+1} in real space (out)
  double *Jorb;              // cleared
  const double2 *tw0;
  int n0, log0, Ng, dim, nc, nvp, rpc, final_pass;
  double inv_ng;
};

// 3. rpc rows per CTA: inverse x transforms of the nc gather spectra, then
// the node records of the rows (as field.cu's k_pack_nodes)
template <typename T>
__global__ void k_f2_rows_pack(RowArgs p, T *__restrict__ nodes, T *__restrict__ nodes_u) {
  extern __shared__ double2 sm[];
  const int n0 = p.n0, rpc = p.rpc, Ng = p.Ng;
  const int row0 = blockIdx.x * rpc;
  const size_t base = (size_t)row0 * n0;
  const int per = rpc * n0;  // points per component in this CTA
  for (int t = threadIdx.x; t < p.nc * per; t += blockDim.x) {
    const int c = t / per, r = t - c * per;
    const int b = r >> p.log0, xx = r & (n0 - 1);
    sm[c * per + (b << p.log0) + brev_n(xx, p.log0)] = p.spec[(size_t)c * Ng + base + r];
  }
  __syncthreads();
  fft_lines(sm, p.nc * rpc, p.log0, p.tw0, true);
  const int d = p.dim;
  for (int r = threadIdx.x; r < per; r += blockDim.x) {
    const size_t g = base + r;
    T *rec = nodes + g * p.nvp;
    for (int c = 0; c < d; c++) rec[c] = (T)(sm[c * per + r].x * p.inv_ng);
    for (int c = 0; c < 3; c++) {
      rec[d + c] = (T)p.A_n[(size_t)c * Ng + g];
      const double a1 = sm[(d + c) * per + r].x * p.inv_ng;
      rec[d + 3 + c] = (T)a1;
      p.A1_real[(size_t)c * Ng + g] = a1;
      p.Jorb[(size_t)c * Ng + g] = 0.0;
    }
    for (int c = d + 6; c < p.nvp; c++) rec[c] = (T)0;
    if (p.final_pass) {
      for (int c = 0; c < 3; c++) nodes_u[g * 4 + c] = (T)(sm[(d + 3 + c) * per + r].x * p.inv_ng);
      nodes_u[g * 4 + 3] = (T)0;
      for (int c = 0; c < p.nc; c++) p.spec[(size_t)c * Ng + g] = sm[c * per + r];
    }
  }
}

struct F1Args {
  const double *jt;                                   // trial current, real (3 comps)
  const double2 *rho, *phi, *psi, *A, *U;             // accepted state spectra
  double2 *rho1, *phi1, *psi1, *A1, *U1;              // candidate n+1 spectra
  double2 *spec;  // final pass: the nc gather fields in real space (times Ng)
  const double *A_n;                                  // A^n in real space
  double *A1_real;                                    // A^{n+1} in real space (out)
  double *Jorb;                                       // cleared
  const double2 *tw0;
  int n0, log0, nc, nvp, project, final_pass;
  double kx_scale, dt, kap2, sigma1, sigma2, inv_ng;
};

// The 1D field step in one CTA: the mode update is that of k_f2_cols_cn with
// k = (kx, 0, 0), the records those of k_f2_rows_pack with d = 1.
template <typename T>
__global__ void k_f1_field(F1Args p, T *__restrict__ nodes, T *__restrict__ nodes_u) {
  extern __shared__ double2 sm[];
  const int n0 = p.n0, Ng = n0, log0 = p.log0;
  double2 *sj = sm;           // 3 lines of n0
  double2 *so = sm + 3 * n0;  // nc lines of n0
  for (int t = threadIdx.x; t < 3 * n0; t += blockDim.x) {
    const int c = t >> log0, x = t & (n0 - 1);
    sj[(c << log0) + brev_n(x, log0)] = make_double2(p.jt[(size_t)c * Ng + x], 0.0);
  }
  __syncthreads();
  fft_lines(sj, 3, log0, p.tw0, false);
  const double2 z = make_double2(0.0, 0.0);
  const double a = 0.5 * p.dt;
  for (int x = threadIdx.x; x < n0; x += blockDim.x) {
    const int xr = brev_n(x, log0);
    const bool nyq = x == n0 / 2;
    if (nyq && p.project) {
      p.rho1[x] = z; p.phi1[x] = z; p.psi1[x] = z;
      for (int c = 0; c < 3; c++) { p.A1[c * (size_t)Ng + x] = z; p.U1[c * (size_t)Ng + x] = z; }
      for (int c = 0; c < p.nc; c++) so[c * n0 + xr] = z;
      continue;
    }
    const int ix = x < n0 / 2 ? x : x - n0;
    const double kx = nyq ? 0.0 : p.kx_scale * ix;
    const double2 j[3] = {sj[x], sj[n0 + x], sj[2 * n0 + x]};
    // continuity: rho' = rho - dt (i k . j)
    const double2 divj = make_double2(-(kx * j[0].y), kx * j[0].x);
    const double2 rho0 = p.rho[x];
    const double2 rho1 = make_double2(rho0.x - p.dt * divj.x, rho0.y - p.dt * divj.y);
    const double2 rhoh = make_double2(0.5 * (rho0.x + rho1.x), 0.5 * (rho0.y + rho1.y));
    const double b = 0.5 * p.dt * p.kap2 * (kx * kx);
    double2 phi1, psi1;
    const double2 phi0 = p.phi[x];
    const double sr = p.dt * p.kap2 * p.sigma1;
    cn_pair(a, b, phi0, p.psi[x], make_double2(sr * rhoh.x, sr * rhoh.y), &phi1, &psi1);
    p.rho1[x] = rho1; p.phi1[x] = phi1; p.psi1[x] = psi1;
    const double2 phih = make_double2(0.5 * (phi0.x + phi1.x), 0.5 * (phi0.y + phi1.y));
    so[xr] = c_i(kx, phih);
    const double sj2 = p.dt * p.kap2 * p.sigma2;
    for (int c = 0; c < 3; c++) {
      const double2 A0 = p.A[c * (size_t)Ng + x], U0 = p.U[c * (size_t)Ng + x];
      double2 A1, U1;
      cn_pair(a, b, A0, U0, make_double2(sj2 * j[c].x, sj2 * j[c].y), &A1, &U1);
      p.A1[c * (size_t)Ng + x] = A1;
      p.U1[c * (size_t)Ng + x] = U1;
      so[(1 + c) * n0 + xr] = A1;
      if (p.nc > 4)
        so[(4 + c) * n0 + xr] = make_double2(0.5 * (U0.x + U1.x), 0.5 * (U0.y + U1.y));
    }
  }
  __syncthreads();
  fft_lines(so, p.nc, log0, p.tw0, true);
  for (int g = threadIdx.x; g < n0; g += blockDim.x) {
    T *rec = nodes + (size_t)g * p.nvp;
    rec[0] = (T)(so[g].x * p.inv_ng);
    for (int c = 0; c < 3; c++) {
      rec[1 + c] = (T)p.A_n[(size_t)c * Ng + g];
      const double a1 = so[(1 + c) * n0 + g].x * p.inv_ng;
      rec[4 + c] = (T)a1;
      p.A1_real[(size_t)c * Ng + g] = a1;
      p.Jorb[(size_t)c * Ng + g] = 0.0;
    }
    for (int c = 7; c < p.nvp; c++) rec[c] = (T)0;
    if (p.final_pass) {
      for (int c = 0; c < 3; c++) nodes_u[g * 4 + c] = (T)(so[(4 + c) * n0 + g].x * p.inv_ng);
      nodes_u[g * 4 + 3] = (T)0;
      for (int c = 0; c < p.nc; c++) p.spec[(size_t)c * Ng + g] = so[c * n0 + g];
    }
  }
}

constexpr int kF1MaxN = 256;  // one CTA beats the multi-launch path up to here

// largest power of two <= v, at least 1
int pow2_floor(long long v) {
  int p = 1;
  while ((long long)p * 2 <= v) p *= 2;
  return p;
}

constexpr size_t kF2MaxSmem = 200 * 1024;

}  // namespace

int field_evaluate(pic_ctx *ctx, const double *jdev, int final_pass) {
  const Geom &g = ctx->g;
  const int Ng = g.Ng;
  const int d = g.dim;
  const int nc = d + 3 + (final_pass ? 3 : 0);
  const int n0 = g.n[0], n1 = d > 1 ? g.n[1] : 1;
  const size_t col_smem = sizeof(double2) * (size_t)(3 + nc) * n1;
  const size_t row_smem = sizeof(double2) * (size_t)nc * n0;
  if (d == 1 && n0 >= 2 && n0 <= kF1MaxN) {
    F1Args p;
    p.jt = jdev;
    p.rho = ctx->rho_h; p.phi = ctx->phi_h; p.psi = ctx->psi_h; p.A = ctx->A_h; p.U = ctx->U_h;
    p.rho1 = ctx->rho1_h; p.phi1 = ctx->phi1_h; p.psi1 = ctx->psi1_h; p.A1 = ctx->A1_h;
    p.U1 = ctx->U1_h;
    p.spec = ctx->work_h;
    p.A_n = ctx->A_real;
    p.A1_real = ctx->A1_real;
    p.Jorb = ctx->Jorb;
    p.tw0 = ctx->tw[0];
    p.n0 = n0; p.log0 = g.logn[0]; p.nc = nc; p.nvp = node_record_len(1);
    p.project = ctx->opt.project_nyquist; p.final_pass = final_pass;
    p.kx_scale = 2.0 * M_PI / g.L[0];
    p.dt = ctx->dt;
    p.kap2 = ctx->opt.kappa * ctx->opt.kappa;
    p.sigma1 = ctx->opt.sigma1;
    p.sigma2 = ctx->opt.sigma2;
    p.inv_ng = 1.0 / Ng;
    const size_t sm = sizeof(double2) * (size_t)(3 + nc) * n0;  // at most 40 KB
    int th = nc * n0 / 2;
    th = th < 64 ? 64 : (th > 256 ? 256 : (th + 31) / 32 * 32);
    if (ctx->eval_f32)
      k_f1_field<float><<<1, th, sm, ctx->st>>>(p, ctx->nodes_f, ctx->nodes_u_f);
    else if (ctx->rsize == 8)
      k_f1_field<double><<<1, th, sm, ctx->st>>>(p, (double *)ctx->nodes, (double *)ctx->nodes_u);
    else
      k_f1_field<float><<<1, th, sm, ctx->st>>>(p, (float *)ctx->nodes, (float *)ctx->nodes_u);
    KCHECK();
    return PIC_OK;
  }
  if (d != 2 || n0 < 2 || n1 < 2 || col_smem > kF2MaxSmem || row_smem > kF2MaxSmem) {
    // the generic path (1D, 3D, very large meshes)
    int e;
    if ((e = field_real_to_complex(ctx, jdev, ctx->jh, 3))) return e;
    if ((e = fft_nd(ctx, ctx->jh, 3, -1))) return e;
    if ((e = field_cn_update(ctx, ctx->jh, final_pass))) return e;
    if ((e = field_pack_nodes(ctx, final_pass))) return e;
    CK(cudaMemsetAsync(ctx->Jorb, 0, sizeof(double) * 3 * Ng, ctx->st));
    return PIC_OK;
  }
  const int log0 = g.logn[0], log1 = g.logn[1];
  // 1. rows: enough CTAs for two waves, whole rows in shared memory
  int rpc = pow2_floor((long long)n1 * 3 / (2LL * ctx->num_sms));
  while (rpc > 1 && (size_t)rpc * n0 * sizeof(double2) > 64 * 1024) rpc /= 2;
  if (rpc > n1) rpc = n1;
  {
    const size_t sm = sizeof(double2) * (size_t)rpc * n0;
    int th = rpc * n0 / 2;
    th = th < 32 ? 32 : (th > 256 ? 256 : (th + 31) / 32 * 32);
    CK(cudaFuncSetAttribute(k_f2_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_f2_rows_fwd<<<dim3(n1 / rpc, 3), th, sm, ctx->st>>>(jdev, ctx->jh, n0, log0, Ng, rpc,
                                                          ctx->tw[0]);
    KCHECK();
  }
  // 2. columns
  {
    ColArgs p;
    p.jh = ctx->jh;
    p.rho = ctx->rho_h; p.phi = ctx->phi_h; p.psi = ctx->psi_h; p.A = ctx->A_h; p.U = ctx->U_h;
    p.rho1 = ctx->rho1_h; p.phi1 = ctx->phi1_h; p.psi1 = ctx->psi1_h; p.A1 = ctx->A1_h;
    p.U1 = ctx->U1_h;
    p.out = ctx->work_h;
    p.tw1 = ctx->tw[1];
    p.n0 = n0; p.n1 = n1; p.log1 = log1; p.Ng = Ng; p.dim = d; p.nc = nc;
    p.project = ctx->opt.project_nyquist;
    p.kx_scale = 2.0 * M_PI / g.L[0];
    p.ky_scale = 2.0 * M_PI / g.L[1];
    p.dt = ctx->dt;
    p.kap2 = ctx->opt.kappa * ctx->opt.kappa;
    p.sigma1 = ctx->opt.sigma1;
    p.sigma2 = ctx->opt.sigma2;
    int th = nc * n1 / 2;
    th = th < 64 ? 64 : (th > 256 ? 256 : (th + 31) / 32 * 32);
    CK(cudaFuncSetAttribute(k_f2_cols_cn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)col_smem));
    k_f2_cols_cn<<<n0, th, col_smem, ctx->st>>>(p);
    KCHECK();
  }
  // 3. rows: inverse x transforms and the node records
  {
    int rpr = pow2_floor((long long)n1 / (2LL * ctx->num_sms));
    while (rpr > 1 && (size_t)rpr * row_smem > 64 * 1024) rpr /= 2;
    if (rpr > n1) rpr = n1;
    RowArgs p;
    p.spec = ctx->work_h;
    p.A_n = ctx->A_real;
    p.A1_real = ctx->A1_real;
    p.Jorb = ctx->Jorb;
    p.tw0 = ctx->tw[0];
    p.n0 = n0; p.log0 = log0; p.Ng = Ng; p.dim = d; p.nc = nc; p.nvp = node_record_len(d);
    p.rpc = rpr; p.final_pass = final_pass; p.inv_ng = 1.0 / Ng;
    const size_t sm = (size_t)rpr * row_smem;
    int th = nc * rpr * n0 / 2;
    th = th < 64 ? 64 : (th > 256 ? 256 : (th + 31) / 32 * 32);
    const int grid = n1 / rpr;
    if (ctx->eval_f32) {  // FP32 records for the FP32 stage of an FP64 context
      CK(cudaFuncSetAttribute(k_f2_rows_pack<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sm));
      k_f2_rows_pack<float><<<grid, th, sm, ctx->st>>>(p, ctx->nodes_f, ctx->nodes_u_f);
    } else if (ctx->rsize == 8) {
      CK(cudaFuncSetAttribute(k_f2_rows_pack<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sm));
      k_f2_rows_pack<double><<<grid, th, sm, ctx->st>>>(p, (double *)ctx->nodes,
                                                         (double *)ctx->nodes_u);
    } else {
      CK(cudaFuncSetAttribute(k_f2_rows_pack<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sm));
      k_f2_rows_pack<float><<<grid, th, sm, ctx->st>>>(p, (float *)ctx->nodes,
                                                        (float *)ctx->nodes_u);
    }
    KCHECK();
  }
  return PIC_OK;
}
