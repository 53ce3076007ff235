// control.cu -- Algorithm 1's outer iteration for one context, decided on
// the device (Sec. 4.5: the tests of Eq. mixed-nonlinear-tests, the type-II
// Anderson update of Eq. anderson-type-two-update with its history rules,
// backtracking, damped Picard, the verifying re-evaluation).
//
// A step's outer iteration is two graph launches with no host round trip:
//   loop graph:   while (cond) { trial current -> map evaluation H(j_t) ->
//                                residual and Gram sums -> controller ->
//                                acceptance copies }
//   verify graph: controller says "verify" ? { the final (diagnostic) map
//                                evaluation at the accepted j -> controller }
// The controller (k_sctl, one CTA) merges the residual sums in a fixed order
// and takes the decisions pic_step's host loop takes, in the same order and
// with the same arithmetic; it ends the loop through the while node's
// condition.  The host reads the outcome once, after both graphs.
#include "pic_internal.cuh"
#include "csum.cuh"

#include <cmath>
#include <cstring>

namespace {

constexpr int kMh = PIC_MAX_ANDERSON;
constexpr int kST = 256;           // threads of the vector kernels and the controller
constexpr int kSMaxBlocks = 512;   // blocks of the residual pass
constexpr int kSMaxPairs = (kMh + 1) * (kMh + 2) / 2 + (kMh + 1);
constexpr int kSStride = 8 + kSMaxPairs;  // doubles of one block's partials

enum { SC_START = 0, SC_TRIAL = 1, SC_VERIFY = 2, SC_DONE = 3, SC_FAILED = 4 };

struct SParams {
  int M, anderson_start, levels, outer_max, growth_scaled, max_rounds;
  double beta, lambda, dc, growth, tr, ta;
  int Ng;
};

}  // namespace

// Controller state of one step (device memory; copied to the host once).
struct SCtl {
  int stage, k, mh, hist0, lvl, attempt, ndir, accept, accept_slot;
  int outer_iters, map_evals, status, rounds, ncol, why;
  int verify_ran;      // the verification evaluation ran
  int col[kMh + 1];    // Gram columns of the trial: ring slots, -1 = the new column
  int dir_slot[kMh];   // columns of the Anderson direction
  double alpha;
  double T_srms, T_smax, T_rms;   // tests of the current iterate
  double res_srms, res_smax;      // tests reported for the step
  double gam[kMh];
  double G[kMh * kMh], g[kMh];    // dR^T dR and dR^T r of the history
  unsigned long long inner_sum, pieces, refined;  // over all evaluations
  unsigned long long map_ns;                      // particle-map device time
  int inner_max_final;
  unsigned long long inner_sum_final, refined_final;
};

namespace {

// jt = j (start, verification) or j + alpha (beta r - sum_c gam_c (dJ_c + beta dR_c))
__global__ void k_strial(const double *__restrict__ j, const double *__restrict__ r,
                         double *__restrict__ jt, const double *__restrict__ dJ,
                         const double *__restrict__ dR, const SCtl *__restrict__ ctl, size_t N3,
                         double beta) {
  const int stage = ctl->stage;
  const double alpha = ctl->alpha;
  const int nd = ctl->ndir;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N3;
       i += (size_t)gridDim.x * blockDim.x) {
    if (stage != SC_TRIAL) {
      jt[i] = j[i];
      continue;
    }
    double s = beta * r[i];
    for (int c = 0; c < nd; c++) {
      const size_t o = (size_t)ctl->dir_slot[c] * N3 + i;
      s -= (dJ[o] + beta * dR[o]) * ctl->gam[c];
    }
    jt[i] = 1.0 * j[i] + alpha * s;
  }
}

// rt = Ht - jt, and per block: compensated |rt|^2, |Ht|^2, |jt|^2, the
// largest scaled node residual, and the Gram products of the columns the
// history would hold if this trial were accepted (ctl->col: ring slots of
// dR, -1 for the new column rt - r), then of each column with rt.  The
// column count NC is a template argument, so that the per-thread products
// stay in registers; kSR-thread blocks, one node per thread.
constexpr int kSR = 128;

template <int NC>
__device__ __forceinline__ void sresid_pass(const double *__restrict__ Ht,
                                            const double *__restrict__ jt,
                                            double *__restrict__ rt,
                                            const double *__restrict__ r,
                                            const double *__restrict__ dR,
                                            const SCtl *__restrict__ ctl, int Ng, double tau_r,
                                            double tau_a, double *__restrict__ parts,
                                            CSum (*sh)[kSR / 32], double *shm,
                                            double (*shp)[kSR / 32]) {
  constexpr int NP = NC * (NC + 1) / 2 + NC;
  int col[NC > 0 ? NC : 1];
#pragma unroll
  for (int a = 0; a < NC; a++) col[a] = ctl->col[a];
  double acc[NP > 0 ? NP : 1];
#pragma unroll
  for (int p = 0; p < NP; p++) acc[p] = 0.0;
  CSum cs[3] = {csum_zero(), csum_zero(), csum_zero()};
  double mx = 0.0;
  const size_t N3 = 3 * (size_t)Ng;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < Ng; g += gridDim.x * blockDim.x) {
    double rr = 0.0, hh = 0.0, jj = 0.0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const size_t i = (size_t)c * Ng + g;
      const double hv = Ht[i], jv = jt[i];
      const double rv = hv - jv;
      rt[i] = rv;
      rr += rv * rv;
      hh += hv * hv;
      jj += jv * jv;
      if (NC > 0) {
        double v[NC > 0 ? NC : 1];
#pragma unroll
        for (int a = 0; a < NC; a++)
          v[a] = col[a] < 0 ? rv - r[i] : dR[(size_t)col[a] * N3 + i];
        int p = 0;
#pragma unroll
        for (int a = 0; a < NC; a++)
#pragma unroll
          for (int b = a; b < NC; b++) acc[p++] += v[a] * v[b];
#pragma unroll
        for (int a = 0; a < NC; a++) acc[p++] += v[a] * rv;
      }
    }
    csum_add(cs[0], rr);
    csum_add(cs[1], hh);
    csum_add(cs[2], jj);
    mx = fmax(mx, sqrt(rr) / (tau_a + 0.5 * tau_r * (sqrt(hh) + sqrt(jj))));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 3; q++) {
    const CSum x = csum_warp(cs[q]);
    if (lane == 0) sh[q][wid] = x;
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if (lane == 0) shm[wid] = mx;
#pragma unroll
  for (int p = 0; p < NP; p++) {
    double x = acc[p];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) shp[p][wid] = x;
  }
  __syncthreads();
  double *out = parts + (size_t)blockIdx.x * kSStride;
  if (threadIdx.x < 3) {
    CSum t = csum_zero();
    for (int w = 0; w < kSR / 32; w++) t = csum_merge(t, sh[threadIdx.x][w]);
    out[2 * threadIdx.x] = t.s;
    out[2 * threadIdx.x + 1] = t.c;
  } else if (threadIdx.x == 3) {
    double m = 0.0;
    for (int w = 0; w < kSR / 32; w++) m = fmax(m, shm[w]);
    out[6] = m;
  } else if (threadIdx.x >= 32 && threadIdx.x < 32 + NP) {
    const int p = threadIdx.x - 32;
    double t = 0.0;
    for (int w = 0; w < kSR / 32; w++) t += shp[p][w];
    out[8 + p] = t;
  }
}

__global__ void __launch_bounds__(kSR)
k_sresid(const double *__restrict__ Ht, const double *__restrict__ jt, double *__restrict__ rt,
         const double *__restrict__ r, const double *__restrict__ dR,
         const SCtl *__restrict__ ctl, int Ng, double tau_r, double tau_a,
         double *__restrict__ parts) {
  __shared__ CSum sh[3][kSR / 32];
  __shared__ double shm[kSR / 32];
  __shared__ double shp[kSMaxPairs][kSR / 32];
  static_assert(kMh + 1 == 9, "one case per Gram column count below");
  static_assert(32 + kSMaxPairs <= kSR, "a thread per Gram product in the block merge");
#define PIC_SRESID(NC)                                                                     \
  case NC:                                                                                 \
    sresid_pass<NC>(Ht, jt, rt, r, dR, ctl, Ng, tau_r, tau_a, parts, sh, shm, shp); \
    break;
  switch (ctl->ncol) {  // the same for every thread
    PIC_SRESID(0)
    PIC_SRESID(1)
    PIC_SRESID(2)
    PIC_SRESID(3)
    PIC_SRESID(4)
    PIC_SRESID(5)
    PIC_SRESID(6)
    PIC_SRESID(7)
    PIC_SRESID(8)
    PIC_SRESID(9)
    default: break;
  }
#undef PIC_SRESID
}

__device__ bool sdev_solve(int m, double *A, double *b) {
  for (int c = 0; c < m; c++) {
    int piv = c;
    for (int r = c + 1; r < m; r++)
      if (fabs(A[r * m + c]) > fabs(A[piv * m + c])) piv = r;
    if (A[piv * m + c] == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < m; k++) {
        const double t = A[c * m + k];
        A[c * m + k] = A[piv * m + k];
        A[piv * m + k] = t;
      }
      const double t = b[c];
      b[c] = b[piv];
      b[piv] = t;
    }
    for (int r = c + 1; r < m; r++) {
      const double f = A[r * m + c] / A[c * m + c];
      for (int k = c; k < m; k++) A[r * m + k] -= f * A[c * m + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = m - 1; c >= 0; c--) {
    double s = b[c];
    for (int k = c + 1; k < m; k++) s -= A[c * m + k] * b[k];
    b[c] = s / A[c * m + c];
    if (!isfinite(b[c])) return false;
  }
  return true;
}

__device__ void s_fail(SCtl &s, int status, int why) {
  s.stage = SC_FAILED;
  s.status = status;
  s.why = why;
}

// the next trial along the current direction, and the Gram columns the
// history would hold if it were accepted
__device__ void s_issue_trial(SCtl &s, const SParams &sp) {
  s.stage = SC_TRIAL;
  s.map_evals++;
  s.ncol = 0;
  if (sp.M > 0) {
    const int keep = s.mh == sp.M ? sp.M - 1 : s.mh;
    const int first = s.mh == sp.M ? s.hist0 + 1 : s.hist0;
    for (int c = 0; c < keep; c++) s.col[c] = (first + c) % sp.M;
    s.col[keep] = -1;
    s.ncol = keep + 1;
  }
}

// the top of an outer iteration: verify, or choose the next direction
__device__ void s_outer_top(SCtl &s, const SParams &sp) {
  s.outer_iters = s.k + 1;
  s.res_srms = s.T_srms;
  s.res_smax = s.T_smax;
  if (s.T_srms <= 1.0 && s.T_smax <= 1.0) {
    s.stage = SC_VERIFY;
    s.ncol = 0;
    s.map_evals++;
    return;
  }
  bool have = false;
  if (s.k + 1 >= sp.anderson_start && s.mh > 0) {  // iterations counted from 1
    const int m = s.mh;
    double A[kMh * kMh], b[kMh], tr_g = 0.0;
    for (int p = 0; p < m; p++) {
      for (int q = 0; q < m; q++) A[p * m + q] = s.G[p * kMh + q];
      b[p] = s.g[p];
      tr_g += A[p * m + p];
    }
    for (int p = 0; p < m; p++) A[p * m + p] += sp.lambda * tr_g / m;
    if (isfinite(tr_g) && tr_g > 0.0 && sdev_solve(m, A, b)) {
      have = true;
      s.ndir = m;
      for (int c = 0; c < m; c++) {
        s.dir_slot[c] = (s.hist0 + c) % sp.M;
        s.gam[c] = b[c];
      }
    } else {
      s.mh = 0;  // unusable history
    }
  }
  if (!have) s.ndir = 0;
  s.attempt = have ? 0 : 1;
  s.lvl = 0;
  s.alpha = 1.0;
  s_issue_trial(s, sp);
}

// Merges the residual pass's block partials (fixed order), then thread 0
// takes Algorithm 1's decision for the evaluation that just ran.
__global__ void __launch_bounds__(kST)
k_sctl(SCtl *__restrict__ ctl, const double *__restrict__ parts, int nb,
       const EvalCounters *__restrict__ cnt, unsigned long long *__restrict__ tim, SParams sp,
       int set_cond, cudaGraphConditionalHandle cond) {
  __shared__ CSum sh[3][kST];
  __shared__ double shm[kST];
  __shared__ double shp[kSMaxPairs];
  const int ncol = ctl->ncol;
  const int npairs = ncol * (ncol + 1) / 2 + ncol;
  for (int q = 0; q < 3; q++) {
    CSum t = csum_zero();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
      t = csum_merge(t, CSum{parts[(size_t)b * kSStride + 2 * q],
                             parts[(size_t)b * kSStride + 2 * q + 1]});
    sh[q][threadIdx.x] = t;
  }
  double m = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = fmax(m, parts[(size_t)b * kSStride + 6]);
  shm[threadIdx.x] = m;
  if ((int)threadIdx.x < npairs) {  // plain sums in block order
    double t = 0.0;
    for (int b = 0; b < nb; b++) t += parts[(size_t)b * kSStride + 8 + threadIdx.x];
    shp[threadIdx.x] = t;
  }
  __syncthreads();
  for (int st = kST / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      for (int q = 0; q < 3; q++)
        sh[q][threadIdx.x] = csum_merge(sh[q][threadIdx.x], sh[q][threadIdx.x + st]);
      shm[threadIdx.x] = fmax(shm[threadIdx.x], shm[threadIdx.x + st]);
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  SCtl &s = *ctl;
  const double n3 = 3.0 * sp.Ng;
  const double rms = sqrt(csum_value(sh[0][0]) / n3);
  const double srms =
      rms / (sp.ta + 0.5 * sp.tr * (sqrt(csum_value(sh[1][0]) / n3) + sqrt(csum_value(sh[2][0]) / n3)));
  const double smax = shm[0];
  const EvalCounters C = *cnt;
  s.inner_sum += C.inner_sum;
  s.pieces += C.pieces;
  s.refined += C.refined;
  if (tim) {
    if (tim[1] > tim[0]) s.map_ns += tim[1] - tim[0];
    tim[0] = ~0ull;
    tim[1] = 0ull;
  }
  s.accept = 0;
  s.accept_slot = -1;
  s.rounds++;
  switch (s.stage) {
    case SC_START:
      if (C.status) { s_fail(s, PIC_EINNER, 1); break; }
      s.accept = 1;
      s.T_srms = srms;
      s.T_smax = smax;
      s.T_rms = rms;
      s.k = 0;
      s_outer_top(s, sp);
      break;
    case SC_TRIAL:
      if (C.status) { s_fail(s, PIC_EINNER, 1); break; }
      if (srms <= (1.0 - sp.dc * s.alpha) * s.T_srms && smax <= sp.growth * s.T_smax) {
        s.accept = 1;
        if (sp.M > 0) {
          int slot;
          if (s.mh == sp.M) {
            slot = s.hist0;
            s.hist0 = (s.hist0 + 1) % sp.M;
          } else {
            slot = (s.hist0 + s.mh) % sp.M;
            s.mh++;
          }
          s.accept_slot = slot;
          int p = 0;
          for (int a = 0; a < ncol; a++)
            for (int b = a; b < ncol; b++, p++) {
              s.G[a * kMh + b] = shp[p];
              s.G[b * kMh + a] = shp[p];
            }
          for (int a = 0; a < ncol; a++) s.g[a] = shp[p++];
          const double grown = sp.growth_scaled ? srms / s.T_srms : rms / s.T_rms;
          if (grown > sp.growth) {
            s.mh = 0;
            s.hist0 = 0;
          }
        }
        s.T_srms = srms;
        s.T_smax = smax;
        s.T_rms = rms;
        s.k++;
        if (s.k >= sp.outer_max) { s_fail(s, PIC_EOUTER, 2); break; }
        s_outer_top(s, sp);
      } else {
        s.lvl++;
        s.alpha *= 0.5;
        if (s.lvl < sp.levels) {
          s_issue_trial(s, sp);
        } else if (s.attempt == 0) {
          s.attempt = 1;
          s.lvl = 0;
          s.alpha = 1.0;
          s.ndir = 0;
          s_issue_trial(s, sp);
        } else {
          s_fail(s, PIC_EOUTER, 3);
        }
      }
      break;
    case SC_VERIFY:
      s.verify_ran = 1;
      if (C.status) { s_fail(s, PIC_EINNER, 1); break; }
      s.res_srms = srms;
      s.res_smax = smax;
      s.inner_max_final = C.inner_max;
      s.inner_sum_final = C.inner_sum;
      s.refined_final = C.refined;
      if (!(srms <= 1.0 && smax <= 1.0)) { s_fail(s, PIC_EOUTER, 4); break; }
      s.stage = SC_DONE;
      s.status = PIC_OK;
      s.accept = 1;
      break;
    default:
      break;
  }
  if (s.stage == SC_TRIAL && s.rounds >= sp.max_rounds) s_fail(s, PIC_EOUTER, 5);
  if (set_cond) cudaGraphSetConditional(cond, s.stage == SC_TRIAL ? 1u : 0u);
}

// the accepted trial becomes the current iterate; its differences enter the
// history slot the controller chose
__global__ void k_saccept(double *__restrict__ j, double *__restrict__ H, double *__restrict__ r,
                          const double *__restrict__ jt, const double *__restrict__ Ht,
                          const double *__restrict__ rt, double *__restrict__ dJ,
                          double *__restrict__ dR, const SCtl *__restrict__ ctl, size_t N3) {
  if (!ctl->accept) return;
  const int slot = ctl->accept_slot;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N3;
       i += (size_t)gridDim.x * blockDim.x) {
    if (slot >= 0) {
      dJ[(size_t)slot * N3 + i] = jt[i] - j[i];
      dR[(size_t)slot * N3 + i] = rt[i] - r[i];
    }
    j[i] = jt[i];
    H[i] = Ht[i];
    r[i] = rt[i];
  }
}

// step start: j = the accepted current (Jacc null: j is kept, a second
// stage continues from the first one's iterate), controller reset
__global__ void k_sinit(double *__restrict__ j, const double *__restrict__ Jacc, size_t N3,
                        SCtl *__restrict__ ctl, unsigned long long *__restrict__ tim) {
  if (Jacc)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N3;
         i += (size_t)gridDim.x * blockDim.x)
      j[i] = Jacc[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    SCtl &s = *ctl;
    s.stage = SC_START;
    s.k = s.mh = s.hist0 = s.lvl = s.attempt = s.ndir = s.accept = 0;
    s.accept_slot = -1;
    s.outer_iters = 0;
    s.map_evals = 1;
    s.status = PIC_OK;
    s.rounds = 0;
    s.ncol = 0;
    s.why = 0;
    s.verify_ran = 0;
    s.alpha = 0.0;
    s.T_srms = s.T_smax = s.T_rms = s.res_srms = s.res_smax = 0.0;
    s.inner_sum = s.pieces = s.refined = s.map_ns = 0ull;
    s.inner_max_final = 0;
    s.inner_sum_final = s.refined_final = 0ull;
    tim[0] = ~0ull;
    tim[1] = 0ull;
  }
}

// condition of the verification: the loop ended with the tests passed
__global__ void k_vcond(const SCtl *__restrict__ ctl, cudaGraphConditionalHandle cond) {
  cudaGraphSetConditional(cond, ctl->stage == SC_VERIFY ? 1u : 0u);
}

int sgrid(size_t n) {
  size_t b = (n + kST - 1) / kST;
  if (b > 1024) b = 1024;
  return (int)(b < 1 ? 1 : b);
}

int sresid_blocks(const pic_ctx *ctx) {
  size_t b = ((size_t)ctx->g.Ng + kSR - 1) / kSR;
  if (b > (size_t)kSMaxBlocks) b = kSMaxBlocks;
  return (int)(b < 1 ? 1 : b);
}

SParams sparams(const pic_ctx *ctx, double tr, double ta) {
  SParams sp;
  sp.M = ctx->opt.anderson_m;
  sp.anderson_start = ctx->opt.anderson_start;
  sp.levels = ctx->opt.backtrack_levels;
  sp.outer_max = ctx->opt.outer_max;
  sp.growth_scaled = ctx->opt.growth_scaled;
  // every round is one evaluation; Algorithm 1 takes at most 1 + outer_max
  // (2 levels + 1) of them before it ends
  sp.max_rounds = 2 + ctx->opt.outer_max * (2 * ctx->opt.backtrack_levels + 1);
  sp.beta = ctx->opt.beta;
  sp.lambda = ctx->opt.lambda;
  sp.dc = ctx->opt.decrease_coef;
  sp.growth = ctx->opt.growth_limit;
  sp.tr = tr;
  sp.ta = ta;
  sp.Ng = ctx->g.Ng;
  return sp;
}

// one evaluation at jt into Ht / rt and the controller's decision on it
int enqueue_round(pic_ctx *ctx, const StepConst &sc, double tr, double ta, int final_pass,
                  int set_cond, cudaGraphConditionalHandle cond) {
  const size_t N3 = 3 * (size_t)ctx->g.Ng;
  int e;
  k_strial<<<sgrid(N3), kST, 0, ctx->st>>>(ctx->j, ctx->r, ctx->jt, ctx->dJ, ctx->dR, ctx->sctl,
                                           N3, ctx->opt.beta);
  KCHECK();
  if ((e = field_evaluate(ctx, ctx->jt, final_pass))) return e;
  if ((e = particles_map_launch(ctx, sc, final_pass))) return e;
  if ((e = field_project_real(ctx, ctx->Jorb, ctx->Ht, 3))) return e;
  const int nb = sresid_blocks(ctx);
  k_sresid<<<nb, kSR, 0, ctx->st>>>(ctx->Ht, ctx->jt, ctx->rt, ctx->r, ctx->dR, ctx->sctl,
                                     ctx->g.Ng, tr, ta, ctx->sred);
  KCHECK();
  k_sctl<<<1, kST, 0, ctx->st>>>(ctx->sctl, ctx->sred, nb, ctx->cnt_dev, ctx->map_timer,
                                 sparams(ctx, tr, ta), set_cond, cond);
  KCHECK();
  k_saccept<<<sgrid(N3), kST, 0, ctx->st>>>(ctx->j, ctx->H, ctx->r, ctx->jt, ctx->Ht, ctx->rt,
                                            ctx->dJ, ctx->dR, ctx->sctl, N3);
  KCHECK();
  return PIC_OK;
}

void destroy_entry(pic_ctx::StepGraphs &g) {
  if (g.loop) cudaGraphExecDestroy(g.loop);
  if (g.verify) cudaGraphExecDestroy(g.verify);
  g.loop = g.verify = nullptr;
}

// Builds the loop and verification graphs of the current buffers and
// tolerances.  False (no error pending) if the driver refuses either.
bool build_step_graphs(pic_ctx *ctx, const StepConst &sc, double tr, double ta,
                       pic_ctx::StepGraphs &out) {
  const long long before = ctx->launches;
  out.loop = out.verify = nullptr;
  // loop graph: one conditional while node
  cudaGraph_t g = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
  cudaGraphConditionalHandle cw = 0;
  if (ok)
    ok = cudaGraphConditionalHandleCreate(&cw, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node = nullptr;
  if (ok) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cw;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
  }
  if (ok) {
    ok = cudaStreamBeginCaptureToGraph(ctx->st, np.conditional.phGraph_out[0], nullptr, nullptr,
                                       0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      ctx->loop_capture = 1;
      const long long b0 = ctx->launches;
      const int e = enqueue_round(ctx, sc, tr, ta, 0, 1, cw);
      out.nk_round = (int)(ctx->launches - b0);
      ctx->loop_capture = 0;
      cudaGraph_t cap = nullptr;
      ok = cudaStreamEndCapture(ctx->st, &cap) == cudaSuccess && e == PIC_OK;
    }
  }
  if (ok) ok = cudaGraphInstantiate(&out.loop, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (ctx->eval_f32) {  // the FP32 stage never verifies: no verification graph
    out.nk_verify = 0;
    ctx->launches = before;
    ctx->loop_capture = 0;
    cudaGetLastError();
    if (!ok) destroy_entry(out);
    return ok;
  }
  // verification graph: the condition kernel, then a conditional if node
  cudaGraph_t g2 = nullptr;
  cudaGraphConditionalHandle cv = 0;
  if (ok) ok = cudaGraphCreate(&g2, 0) == cudaSuccess;
  if (ok)
    ok = cudaGraphConditionalHandleCreate(&cv, g2, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNode_t knode = nullptr;
  if (ok) {
    ok = cudaStreamBeginCaptureToGraph(ctx->st, g2, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      k_vcond<<<1, 1, 0, ctx->st>>>(ctx->sctl, cv);
      const bool lok = cudaGetLastError() == cudaSuccess;
      cudaGraph_t cap = nullptr;
      ok = cudaStreamEndCapture(ctx->st, &cap) == cudaSuccess && lok;
    }
    size_t n = 1;
    if (ok) ok = cudaGraphGetNodes(g2, &knode, &n) == cudaSuccess && n == 1;
  }
  cudaGraphNodeParams np2 = {};
  cudaGraphNode_t inode = nullptr;
  if (ok) {
    np2.type = cudaGraphNodeTypeConditional;
    np2.conditional.handle = cv;
    np2.conditional.type = cudaGraphCondTypeIf;
    np2.conditional.size = 1;
    ok = cudaGraphAddNode(&inode, g2, &knode, nullptr, 1, &np2) == cudaSuccess;
  }
  if (ok) {
    ok = cudaStreamBeginCaptureToGraph(ctx->st, np2.conditional.phGraph_out[0], nullptr, nullptr,
                                       0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      ctx->loop_capture = 1;
      const long long b0 = ctx->launches;
      const int e = enqueue_round(ctx, sc, tr, ta, 1, 0, 0);
      out.nk_verify = 1 + (int)(ctx->launches - b0);
      ctx->loop_capture = 0;
      cudaGraph_t cap = nullptr;
      ok = cudaStreamEndCapture(ctx->st, &cap) == cudaSuccess && e == PIC_OK;
    }
  }
  if (ok) ok = cudaGraphInstantiate(&out.verify, g2, 0) == cudaSuccess;
  if (g2) cudaGraphDestroy(g2);
  ctx->launches = before;
  ctx->loop_capture = 0;
  cudaGetLastError();  // a refused build falls back to the host-driven step
  if (!ok) destroy_entry(out);
  return ok;
}

}  // namespace

int control_alloc(pic_ctx *ctx) {
  CK(cudaMalloc((void **)&ctx->sctl, sizeof(SCtl)));
  CK(cudaMemset(ctx->sctl, 0, sizeof(SCtl)));
  CK(cudaMallocHost((void **)&ctx->sctl_host, sizeof(SCtl)));
  CK(cudaMalloc((void **)&ctx->map_timer, 2 * sizeof(unsigned long long)));
  CK(cudaMalloc((void **)&ctx->sred, sizeof(double) * kSStride * kSMaxBlocks));
  return PIC_OK;
}

void control_graphs_clear(pic_ctx *ctx) {
  for (int k = 0; k < ctx->nsgraphs; k++) destroy_entry(ctx->sgraphs[k]);
  ctx->nsgraphs = 0;
}

void control_free(pic_ctx *ctx) {
  control_graphs_clear(ctx);
  if (ctx->sctl) cudaFree(ctx->sctl);
  if (ctx->sctl_host) cudaFreeHost(ctx->sctl_host);
  if (ctx->map_timer) cudaFree(ctx->map_timer);
  if (ctx->sred) cudaFree(ctx->sred);
  ctx->sctl = nullptr;
  ctx->sctl_host = nullptr;
  ctx->map_timer = nullptr;
  ctx->sred = nullptr;
}

int step_control_device(pic_ctx *ctx, const StepConst &sc, double tr, double ta, StepOutcome *out,
                        int *ran, int from_j, int verify) {
  *ran = 0;
  if (ctx->sgraphs_off || ctx->graphs_off || ctx->np == 0 || !ctx->sctl ||
      (ctx->eval_f32 && ctx->f32_stage_off) || (verify && ctx->eval_f32))
    return PIC_OK;
  pic_ctx::StepGraphs *ent = nullptr;
  for (int k = 0; k < ctx->nsgraphs; k++) {
    pic_ctx::StepGraphs &g = ctx->sgraphs[k];
    if (g.phi == ctx->phi_h && g.A == ctx->A_real && g.tr == tr && g.ta == ta &&
        g.itr == sc.tau_r && g.ita == sc.tau_a && g.np == ctx->np && g.f32 == ctx->eval_f32) {
      ent = &g;
      break;
    }
  }
  if (!ent) {
    if (ctx->nsgraphs == 4) control_graphs_clear(ctx);
    pic_ctx::StepGraphs &g = ctx->sgraphs[ctx->nsgraphs];
    if (!build_step_graphs(ctx, sc, tr, ta, g)) {
      // the host drives the step; a refused FP32-stage graph only drops
      // the FP32 stage
      if (ctx->eval_f32) ctx->f32_stage_off = 1;
      else ctx->sgraphs_off = 1;
      return PIC_OK;
    }
    g.phi = ctx->phi_h;
    g.A = ctx->A_real;
    g.tr = tr;
    g.ta = ta;
    g.itr = sc.tau_r;
    g.ita = sc.tau_a;
    g.np = ctx->np;
    g.f32 = ctx->eval_f32;
    ctx->nsgraphs++;
    ent = &g;
  }
  *ran = 1;
  const size_t N3 = 3 * (size_t)ctx->g.Ng;
  k_sinit<<<sgrid(N3), kST, 0, ctx->st>>>(ctx->j, from_j ? nullptr : ctx->J_acc, N3, ctx->sctl,
                                          ctx->map_timer);
  KCHECK();
  CK(cudaGraphLaunch(ent->loop, ctx->st));
  if (verify) CK(cudaGraphLaunch(ent->verify, ctx->st));
  CK(cudaMemcpyAsync(ctx->sctl_host, ctx->sctl, sizeof(SCtl), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  const SCtl &s = *ctx->sctl_host;
  const bool verified = s.verify_ran != 0;
  const int loop_rounds = s.rounds - (verified ? 1 : 0);
  ctx->launches += (long long)ent->nk_round * loop_rounds + (verified ? ent->nk_verify : verify);
  ctx->map_launches += s.map_evals;
  ctx->map_ms += 1e-6 * (double)s.map_ns;
  ctx->pushes += (long long)ctx->np * s.map_evals;
  ctx->inner_iters += (long long)s.inner_sum;
  ctx->pieces += (long long)s.pieces;
  ctx->refined += (long long)s.refined;
  out->converged = s.stage == SC_VERIFY || s.stage == SC_DONE;  // the tests passed
  out->status = s.stage == SC_DONE ? PIC_OK : s.status;
  out->why = s.why;
  out->outer_iters = s.outer_iters;
  out->map_evals = s.map_evals;
  out->res_srms = s.res_srms;
  out->res_smax = s.res_smax;
  out->inner_max = s.inner_max_final;
  out->inner_sum = s.inner_sum_final;
  out->refined = s.refined_final;
  out->work_p = out->chain = 0.0;
  if (s.stage == SC_DONE) particles_final_sums(ctx, &out->work_p, &out->chain);
  return PIC_OK;
}
