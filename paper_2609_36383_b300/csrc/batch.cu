// batch.cu -- an ensemble of independent 1D3V problems advanced together
// (pic_batch_*): one launch per phase of Algorithm 1 covers every instance,
// and the outer solver's decisions are taken on the device, so a step needs
// no host round trip per map evaluation.
//
// One round of the step is the fixed kernel sequence
//   k_bctl     one thread per instance: reads the results of the previous
//              evaluation (test sums, Gram products, inner counters) and
//              takes the next decision of Algorithm 1 -- accept, backtrack
//              (alpha = 1 .. 2^-(levels-1)), fall back from the Anderson
//              direction to damped Picard, verify, finish or fail -- then
//              sets up the next evaluation of that instance (or none);
//   k_baccept  one CTA per instance: the accepted trial becomes (j, r, H) and
//              enters the Anderson history (dJ, dR);
//   k_btrial   one CTA per instance: trial current j + alpha dir with
//              dir = beta r - sum_c gamma_c (dJ_c + beta dR_c) (Eq.
//              anderson-type-two-update; gamma = 0 for damped Picard);
//   k_bfield   one CTA per instance: the whole spectral field step (Sec. 2.3)
//              in shared memory: FFT of the trial current, Nyquist projection
//              (Eq. nyquist-projector), continuity and the per-mode CN update,
//              inverse FFTs, and the gather records of the particle map;
//   k_bmap     the particle map (inner Picard iteration, GM-HC push, orbit
//              deposit) of map_device.cuh over the blocks of the instances
//              that evaluate: k_bctl lists them, and a persistent grid walks
//              the list, each block reading its instance's geometry (one
//              launch for plain evaluations, one for the final pass);
//   k_bresid   one CTA per instance: H = P J_orb, r = H - j, the sums of Eq.
//              mixed-nonlinear-tests, the Gram products the next Anderson
//              solve needs, and (final pass) the particle and mesh work.
// A step is one CUDA graph launch for all its rounds: a conditional while
// node repeats the round, and k_bctl clears the node's condition once no
// instance evaluates (or at a round limit that Algorithm 1 cannot reach), so
// the host waits once per step.  Instances that finished early skip the rest
// of the rounds.  Where the driver cannot build that graph, the host launches
// the rounds itself and reads the loop state after each.  Every instance
// then commits (or, on failure, keeps) its state exactly as a single-problem
// context does (pic_step).
//
// Per-instance initial states (pic_start) are prepared by a temporary
// single-problem context per distinct grid and copied in.
#include "map_device.cuh"
#include "csum.cuh"
#include "trace.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

namespace {

constexpr int kBT = 256;        // threads of the per-instance kernels
constexpr int kNmax = 1024;     // largest mesh of an instance
constexpr int kMh = PIC_MAX_ANDERSON;
constexpr int kNDots = (kMh + 1) * (kMh + 2) / 2;  // products of <= kMh columns and r
constexpr int kCtlThreads = 1024;

enum BMode { B_IDLE = 0, B_EVAL = 1, B_FINAL = 2 };
enum BPhase { B_RUNNING = 0, B_DONE = 1, B_FAILED = 2 };
enum BStage { S_START = 0, S_INIT = 1, S_TRIAL = 2, S_VERIFY = 3 };
enum BWhy { W_NONE = 0, W_INNER = 1, W_LIMIT = 2, W_NODIR = 3, W_VERIFY = 4 };

struct BInst {
  int nx, logn;
  int64_t moff;        // first mesh node of the instance
  int64_t pbeg, pend;  // particle range; pbeg is a multiple of kPT
  int blk0, nblk;      // particle-kernel blocks of the instance
  int64_t sort_shift;  // pbeg minus the particles of the instances before it
  double L, x0, dx;
};

// Algorithm 1 state of one instance and the set-up of its next evaluation.
struct BState {
  // next round (written by k_bctl, read by the other round kernels)
  int mode, seed, accept, accept_slot;
  int ndir, dir_slot[kMh];
  double alpha, beta, gam[kMh];
  int ncol, col[kMh];  // columns of the Gram products, oldest first (-1: new)
  // outer solver
  int phase, stage, status, why;
  int k, attempt, lvl, mh, hist0;
  double T_srms, T_smax, T_rms;
  double G[kMh * kMh], g[kMh];  // Gram matrix of the history and its products with r
  // report
  int outer_iters, map_evals, inner_max;
  unsigned long long inner_sum, inner_total, pieces_total, refined_total, refined_final;
  double res_srms, res_smax, work_p, chain, work_mesh;
};

// results of one evaluation of one instance
struct BRes {
  double r2, h2, j2, smax;
  double dots[kNDots];
  double work_mesh, work_p, chain;
};

// progress of the round loop of one step (device-resident)
struct BLoop {
  int running;   // instances that evaluate in the current round
  int rounds;    // rounds started in this step
  int overflow;  // the round limit was reached with instances still running
  int nwork[2];  // particle-map blocks of this round: plain evaluations, final passes
  int pad;
};

struct BParams {  // solver constants of the batch
  int M, anderson_start, levels, outer_max, growth_scaled;
  double beta, lambda, dc, growth;
  double tr, ta;  // outer tolerances
};

}  // namespace

struct pic_batch {
  int B;
  int nspecies;
  double qs[PIC_MAX_SPECIES], ms[PIC_MAX_SPECIES];
  double dt;
  pic_options opt;
  cudaStream_t st, own_st;
  int rsize;
  std::string err;
  std::vector<BInst> inst;
  std::vector<int64_t> np;
  std::vector<double> E0;
  int64_t M;    // mesh nodes of all instances
  int64_t cap;  // particle slots (ranges padded to kPT)
  int nblocks;
  int started;
  long long steps_done;
  // staged host inputs (pic_batch_set_instance), consumed by pic_batch_start
  struct Stage {
    std::vector<int32_t> sp;
    std::vector<double> x, u, w, A, U;
    bool set = false;
  };
  std::vector<Stage> stage;
  // device tables
  BInst *d_inst;
  PGeom *d_pg;
  void *d_invdx;  // per instance (1/dx, 1/dV) in the particle type
  int32_t *d_blk2inst;
  int32_t *d_work;  // per-round particle-map block lists (2 x nblocks)
  int num_sms;
  BState *d_state, *h_state;  // h_state pinned
  BRes *d_res;
  EvalCounters *d_cnt;
  BLoop *d_loop, *h_loop;  // h_loop pinned
  // particles
  int32_t *cell, *sp, *iters, *keys, *cnt_sort;
  int64_t *id, *slot;
  void *off, *P, *Am, *v0, *vbar, *Pnew, *tmp_r;
  double *w;
  double *psum;
  // mesh: instance b holds scalars at [moff, moff + nx) and vectors at
  // [3 moff, 3 moff + 3 nx), component-major
  double2 *phi_h, *psi_h, *rho_h, *A_h, *U_h, *phi1_h, *psi1_h, *rho1_h, *A1_h, *U1_h;
  double *A_real, *A1_real, *J_acc, *Jorb, *j, *jt, *H, *Ht, *r, *rt, *Eh, *dJ, *dR;
  void *AT;  // A^n in the particle type (aliases A_real for FP64)
  void *nodes, *nodes_u;
  double2 *tw;
  double *d_diag, *h_diag;  // per instance: K, W, gauss, lorenz (pinned host copy)
  double *d_out;            // export scratch
  // execution: the rounds of a step run as one graph whose while node
  // repeats the round until the controller reports no instance running
  cudaGraphExec_t loop_exec;
  double graph_tr, graph_ta, graph_itr, graph_ita;
  int graph_ok;  // 1 built, 0 not yet, -1 unavailable: host-driven rounds
  long long launches, map_launches, pushes, inner_iters, pieces, refined;
};

namespace {

#define BCK(call)                                                              \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      bt->err = std::string(#call) + ": " + cudaGetErrorString(e_);            \
      return PIC_ECUDA;                                                        \
    }                                                                          \
  } while (0)

#define BKCHECK()                                                              \
  do {                                                                         \
    bt->launches++;                                                            \
    BCK(cudaGetLastError());                                                   \
  } while (0)

__device__ __forceinline__ double2 cmi(double s, double2 z) { return make_double2(-s * z.y, s * z.x); }
__device__ __forceinline__ int brev(int k, int logN) {
  return logN ? (int)(__brev((unsigned)k) >> (32 - logN)) : 0;
}

// In-place iterative radix-2 DIT FFT of ncomp lines of length N held in
// bit-reversed order in shared memory; sign -1 (forward) or +1 (inverse, the
// conjugate twiddles), unnormalised.  tw[m] = exp(-2 pi i m / kNmax).
__device__ void smem_fft(double2 *a, int ncomp, int N, const double2 *__restrict__ tw, int inverse) {
  const int half = N >> 1;
  for (int h = 1; h < N; h <<= 1) {
    const int tstep = kNmax / (2 * h);
    for (int t = threadIdx.x; t < ncomp * half; t += blockDim.x) {
      const int c = t / half, jj = t - c * half;
      const int grp = jj / h, pos = jj - grp * h;
      const int i0 = c * N + grp * 2 * h + pos, i1 = i0 + h;
      double2 wv = tw[pos * tstep];
      if (inverse) wv.y = -wv.y;
      const double2 x0 = a[i0], x1 = a[i1];
      const double2 y = make_double2(wv.x * x1.x - wv.y * x1.y, wv.x * x1.y + wv.y * x1.x);
      a[i0] = make_double2(x0.x + y.x, x0.y + y.y);
      a[i1] = make_double2(x0.x - y.x, x0.y - y.y);
    }
    __syncthreads();
  }
}

// bit-reversal permutation of ncomp lines in place
__device__ void smem_bitrev(double2 *a, int ncomp, int N, int logN) {
  for (int t = threadIdx.x; t < ncomp * N; t += blockDim.x) {
    const int c = t / N, k = t - c * N, kr = brev(k, logN);
    if (k < kr) {
      const double2 v = a[c * N + k];
      a[c * N + k] = a[c * N + kr];
      a[c * N + kr] = v;
    }
  }
  __syncthreads();
}

__device__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w];
  return s;
}

// compensated block sum (every addition a TwoSum; the total in every thread)
__device__ CSum block_csum(CSum v, CSum *sh) {
  v = csum_warp(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  CSum s = csum_zero();
  for (int w = 0; w < (int)(blockDim.x >> 5); w++) s = csum_merge(s, sh[w]);
  return s;
}

__device__ double block_max(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); w++) s = fmax(s, sh[w]);
  return s;
}

// ---- the outer controller ---------------------------------------------------

// Gaussian elimination with partial pivoting on an m x m system (m <= kMh);
// false when singular or not finite
__device__ bool dev_solve(int m, double *A, double *b) {
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

// set up a trial evaluation along the current direction (alpha, gam, ndir)
// and the Gram columns of the history it would produce if accepted
__device__ void issue_trial(BState &s, const BParams &bp) {
  s.mode = B_EVAL;
  s.stage = S_TRIAL;
  s.map_evals++;
  s.ncol = 0;
  if (bp.M > 0) {
    const int keep = s.mh == bp.M ? bp.M - 1 : s.mh;
    const int first = s.mh == bp.M ? s.hist0 + 1 : s.hist0;
    for (int c = 0; c < keep; c++) s.col[c] = (first + c) % bp.M;
    s.col[keep] = -1;
    s.ncol = keep + 1;
  }
}

__device__ void fail(BState &s, int status, int why) {
  s.phase = B_FAILED;
  s.status = status;
  s.why = why;
  s.mode = B_IDLE;
}

// the top of an outer iteration: verify, or pick the next direction
__device__ void outer_top(BState &s, const BParams &bp) {
  s.outer_iters = s.k + 1;
  s.res_srms = s.T_srms;
  s.res_smax = s.T_smax;
  if (s.T_srms <= 1.0 && s.T_smax <= 1.0) {
    s.mode = B_FINAL;
    s.stage = S_VERIFY;
    s.alpha = 0.0;
    s.ndir = 0;
    s.ncol = 0;
    s.map_evals++;
    return;
  }
  bool have = false;
  if (s.k + 1 >= bp.anderson_start && s.mh > 0) {  // iterations counted from 1
    const int m = s.mh;
    double A[kMh * kMh], b[kMh], tr_g = 0.0;
    for (int p = 0; p < m; p++) {
      for (int q = 0; q < m; q++) A[p * m + q] = s.G[p * kMh + q];
      b[p] = s.g[p];
      tr_g += A[p * m + p];
    }
    for (int p = 0; p < m; p++) A[p * m + p] += bp.lambda * tr_g / m;
    if (isfinite(tr_g) && tr_g > 0.0 && dev_solve(m, A, b)) {
      have = true;
      s.ndir = m;
      for (int c = 0; c < m; c++) {
        s.dir_slot[c] = (s.hist0 + c) % bp.M;
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
  s.beta = bp.beta;
  issue_trial(s, bp);
}

// One thread per instance; a single CTA so that it can also count the
// instances still running.
__global__ void __launch_bounds__(kCtlThreads)
k_bctl(int B, BState *__restrict__ states, const BRes *__restrict__ res,
       const EvalCounters *__restrict__ cnts, const BInst *__restrict__ inst, BParams bp,
       BLoop *__restrict__ loop, int max_rounds, cudaGraphConditionalHandle cond,
       int32_t *__restrict__ work, int nblocks) {
  __shared__ int s_run;
  __shared__ int s_cnt[2][kCtlThreads];
  if (threadIdx.x == 0) s_run = 0;
  __syncthreads();
  int run = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    BState &s = states[b];  // worked on in place: the state is too large for registers
    s.accept = 0;
    s.seed = 0;
    if (s.phase != B_RUNNING) {
      s.mode = B_IDLE;
      continue;
    }
    const BRes R = res[b];
    const EvalCounters C = cnts[b];
    const double n3 = 3.0 * inst[b].nx;
    const double rms = sqrt(R.r2 / n3);
    const double srms = rms / (bp.ta + 0.5 * bp.tr * (sqrt(R.h2 / n3) + sqrt(R.j2 / n3)));
    const double smax = R.smax;
    if (s.stage != S_START) {
      s.inner_total += C.inner_sum;
      s.pieces_total += C.pieces;
      s.refined_total += C.refined;
    }
    switch (s.stage) {
      case S_START:
        s.mode = B_EVAL;
        s.seed = 1;
        s.alpha = 0.0;
        s.beta = 0.0;
        s.ndir = 0;
        s.ncol = 0;
        s.map_evals = 1;
        s.stage = S_INIT;
        break;
      case S_INIT:
        if (C.status) { fail(s, PIC_EINNER, W_INNER); break; }
        s.accept = 1;
        s.accept_slot = -1;
        s.T_srms = srms;
        s.T_smax = smax;
        s.T_rms = rms;
        s.k = 0;
        outer_top(s, bp);
        break;
      case S_TRIAL:
        if (C.status) { fail(s, PIC_EINNER, W_INNER); break; }
        if (srms <= (1.0 - bp.dc * s.alpha) * s.T_srms && smax <= bp.growth * s.T_smax) {
          s.accept = 1;
          s.accept_slot = -1;
          if (bp.M > 0) {
            int slot;
            if (s.mh == bp.M) {
              slot = s.hist0;
              s.hist0 = (s.hist0 + 1) % bp.M;
            } else {
              slot = (s.hist0 + s.mh) % bp.M;
              s.mh++;
            }
            s.accept_slot = slot;
            // Gram products of the new history: k_bresid computed them for
            // the columns listed in s.col, then r
            const int nc = s.ncol;
            int d = 0;
            for (int a = 0; a <= nc; a++)
              for (int c = a; c <= nc; c++, d++) {
                const double v = R.dots[d];
                if (c < nc) {
                  s.G[a * kMh + c] = v;
                  s.G[c * kMh + a] = v;
                } else {
                  s.g[a] = v;
                }
              }
            const double grown = bp.growth_scaled ? srms / s.T_srms : rms / s.T_rms;
            if (grown > bp.growth) { s.mh = 0; s.hist0 = 0; }
          }
          s.T_srms = srms;
          s.T_smax = smax;
          s.T_rms = rms;
          s.k++;
          if (s.k >= bp.outer_max) { fail(s, PIC_EOUTER, W_LIMIT); break; }
          outer_top(s, bp);
        } else {
          s.lvl++;
          s.alpha *= 0.5;
          if (s.lvl < bp.levels) {
            issue_trial(s, bp);
          } else if (s.attempt == 0) {
            s.attempt = 1;
            s.lvl = 0;
            s.alpha = 1.0;
            s.ndir = 0;
            issue_trial(s, bp);
          } else {
            fail(s, PIC_EOUTER, W_NODIR);
          }
        }
        break;
      case S_VERIFY:
        if (C.status) { fail(s, PIC_EINNER, W_INNER); break; }
        s.res_srms = srms;
        s.res_smax = smax;
        if (!(srms <= 1.0 && smax <= 1.0)) { fail(s, PIC_EOUTER, W_VERIFY); break; }
        s.phase = B_DONE;
        s.status = PIC_OK;
        s.mode = B_IDLE;
        s.work_p = R.work_p;
        s.chain = R.chain;
        s.work_mesh = R.work_mesh;
        s.inner_max = C.inner_max;
        s.inner_sum = C.inner_sum;
        s.refined_final = C.refined;
        break;
    }
    if (s.phase == B_RUNNING && s.mode != B_IDLE) run++;
  }
  atomicAdd(&s_run, run);
  __syncthreads();
  if (threadIdx.x == 0) {
    // the loop ends when no instance evaluates, or (never expected: Algorithm
    // 1 takes at most 2 + outer_max (2 levels + 1) evaluations) at the limit
    const int r = loop->rounds + 1;
    loop->rounds = r;
    loop->running = s_run;
    const bool more = s_run > 0 && r < max_rounds;
    if (s_run > 0 && !more) loop->overflow = 1;
    if (cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
  }
  // Work lists of this round's particle-map launches: the blocks of the
  // instances that evaluate (list 0: plain evaluations, list 1: final
  // passes), instances in order; each thread lists a contiguous run of
  // instances at offsets from a scan of the counts.
  const int chunk = (B + (int)blockDim.x - 1) / (int)blockDim.x;
  const int b0 = min(B, (int)threadIdx.x * chunk), b1 = min(B, b0 + chunk);
  int c0 = 0, c1 = 0;
  for (int b = b0; b < b1; b++) {
    const int m = states[b].mode;
    if (m == B_EVAL) c0 += inst[b].nblk;
    else if (m == B_FINAL) c1 += inst[b].nblk;
  }
  s_cnt[0][threadIdx.x] = c0;
  s_cnt[1][threadIdx.x] = c1;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {  // inclusive scan of both counts
    const int a0 = (int)threadIdx.x >= o ? s_cnt[0][threadIdx.x - o] : 0;
    const int a1 = (int)threadIdx.x >= o ? s_cnt[1][threadIdx.x - o] : 0;
    __syncthreads();
    s_cnt[0][threadIdx.x] += a0;
    s_cnt[1][threadIdx.x] += a1;
    __syncthreads();
  }
  int o0 = s_cnt[0][threadIdx.x] - c0, o1 = s_cnt[1][threadIdx.x] - c1;
  for (int b = b0; b < b1; b++) {
    const int m = states[b].mode;
    if (m != B_EVAL && m != B_FINAL) continue;
    const BInst in = inst[b];
    int32_t *dst = m == B_EVAL ? work + o0 : work + nblocks + o1;
    for (int k = 0; k < in.nblk; k++) dst[k] = in.blk0 + k;
    if (m == B_EVAL) o0 += in.nblk;
    else o1 += in.nblk;
  }
  if (threadIdx.x == blockDim.x - 1) {
    loop->nwork[0] = s_cnt[0][threadIdx.x];
    loop->nwork[1] = s_cnt[1][threadIdx.x];
  }
}

// start of a step: every instance runs Algorithm 1 from its first evaluation
__global__ void k_bbegin(int B, BState *states, BLoop *loop) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) {
    loop->running = B;
    loop->rounds = 0;
    loop->overflow = 0;
  }
  if (b >= B) return;
  BState s;
  memset(&s, 0, sizeof s);
  s.phase = B_RUNNING;
  s.stage = S_START;
  s.mode = B_IDLE;
  s.status = PIC_OK;
  states[b] = s;
}

// ---- per-instance mesh kernels ------------------------------------------------

struct BMesh {
  const BInst *inst;
  const BState *st;
  double *j, *jt, *H, *Ht, *r, *rt, *dJ, *dR, *Jorb, *Eh, *J_acc;
  int64_t M3;  // stride of a history slot
  BRes *res;
  EvalCounters *cnt;
  const double *psum;
};

// accepted trial: history column (slot >= 0) and (j, r, H) <- trial
__global__ void __launch_bounds__(kBT) k_baccept(BMesh p) {
  const int b = blockIdx.x;
  const BState &s = p.st[b];
  if (!s.accept) return;
  const int slot = s.accept_slot;
  const BInst in = p.inst[b];
  const int64_t base = 3 * in.moff, n3 = 3 * (int64_t)in.nx;
  for (int64_t e = threadIdx.x; e < n3; e += blockDim.x) {
    const int64_t q = base + e;
    if (slot >= 0) {
      p.dJ[slot * p.M3 + q] = p.jt[q] - p.j[q];
      p.dR[slot * p.M3 + q] = p.rt[q] - p.r[q];
    }
    p.j[q] = p.jt[q];
    p.r[q] = p.rt[q];
    p.H[q] = p.Ht[q];
  }
}

// trial current j_t = j + alpha (beta r - sum_c gamma_c (dJ_c + beta dR_c));
// the first evaluation of a step (seed) starts from the accepted current.
// Also clears the instance's inner counters for the coming evaluation.
__global__ void __launch_bounds__(kBT) k_btrial(BMesh p) {
  const int b = blockIdx.x;
  const BState &s = p.st[b];
  if (s.mode == B_IDLE) return;
  if (threadIdx.x == 0) {
    EvalCounters z;
    z.status = 0;
    z.inner_max = 0;
    z.inner_sum = 0;
    z.pieces = 0;
    z.refined = 0;
    p.cnt[b] = z;
  }
  const BInst in = p.inst[b];
  const int64_t base = 3 * in.moff, n3 = 3 * (int64_t)in.nx;
  const double alpha = s.alpha, beta = s.beta;
  const int nd = s.ndir;
  for (int64_t e = threadIdx.x; e < n3; e += blockDim.x) {
    const int64_t q = base + e;
    if (s.seed) {
      const double v = p.J_acc[q];
      p.j[q] = v;
      p.jt[q] = v;
      continue;
    }
    double d = beta * p.r[q];
    for (int c = 0; c < nd; c++) {
      const int64_t sl = s.dir_slot[c];
      d -= (p.dJ[sl * p.M3 + q] + beta * p.dR[sl * p.M3 + q]) * s.gam[c];
    }
    p.jt[q] = p.j[q] + alpha * d;
  }
}

struct BField {
  const BInst *inst;
  const BState *st;
  const double *jt, *A_real;
  const double2 *rho, *phi, *psi, *A, *U;
  double2 *rho1, *phi1, *psi1, *A1, *U1;
  double *A1_real, *Jorb, *Eh;
  const double2 *tw;
  double dt, kap2, sigma1, sigma2;
  int project;
};

// The spectral field step of one instance (Sec. 2.3, Eq. CN-field): with
// a = dt/2, b = dt kappa^2 k^2 / 2 and source s, every mode solves
//   psi' = ((1 - a b) psi - 2 b phi + s) / (1 + a b),  phi' = phi + a (psi' + psi),
// with s = dt kappa^2 sigma1 rho^{1/2} for (phi, psi), where rho' = rho - dt i k j_x
// (continuity), and s = dt kappa^2 sigma2 j_c for (A_c, U_c).  Then the
// gather records [d_x phi^{1/2}, A^n (3), A^{n+1} (3), 0] of every node, and
// on the final pass U^{n+1/2} and E^{n+1/2} = -d_x phi^{1/2} e_x - U^{n+1/2}.
template <typename T>
__global__ void __launch_bounds__(kBT) k_bfield(BField p, T *__restrict__ nodes,
                                                T *__restrict__ nodes_u) {
  extern __shared__ double2 sm[];
  const int b = blockIdx.x;
  const int mode = p.st[b].mode;
  if (mode == B_IDLE) return;
  const BInst in = p.inst[b];
  const int N = in.nx, logN = in.logn;
  const int64_t mo = in.moff;
  const double twopiL = 2.0 * M_PI / in.L;
  for (int t = threadIdx.x; t < 3 * N; t += blockDim.x) {
    const int c = t / N, g = t - c * N;
    sm[c * N + brev(g, logN)] = make_double2(p.jt[3 * mo + t], 0.0);
    p.Jorb[3 * mo + t] = 0.0;  // the deposit target of this evaluation
  }
  __syncthreads();
  smem_fft(sm, 3, N, p.tw, 0);
  const int nout = mode == B_FINAL ? 7 : 4;  // i k phi^{1/2}, A^{n+1} (3), U^{n+1/2} (3)
  const double2 z = make_double2(0.0, 0.0);
  // each mode is read and rewritten by the same thread
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const bool nyq = k == N / 2;
    const bool zero = nyq && p.project;
    const int kk = k < N / 2 ? k : k - N;
    const double kx = nyq ? 0.0 : twopiL * kk;
    double2 jm[3];
    for (int c = 0; c < 3; c++) jm[c] = zero ? z : sm[c * N + k];
    const double2 rho0 = p.rho[mo + k];
    double2 rho1 = make_double2(rho0.x + p.dt * kx * jm[0].y, rho0.y - p.dt * kx * jm[0].x);
    const double2 rhoh = make_double2(0.5 * (rho0.x + rho1.x), 0.5 * (rho0.y + rho1.y));
    const double a = 0.5 * p.dt, bb = 0.5 * p.dt * p.kap2 * kx * kx;
    const double inv = 1.0 / (1.0 + a * bb), c1 = (1.0 - a * bb) * inv, c2 = -2.0 * bb * inv;
    const double2 phi0 = p.phi[mo + k], psi0 = p.psi[mo + k];
    const double s1 = p.dt * p.kap2 * p.sigma1;
    double2 psi1 = make_double2(c1 * psi0.x + c2 * phi0.x + s1 * rhoh.x * inv,
                                c1 * psi0.y + c2 * phi0.y + s1 * rhoh.y * inv);
    double2 phi1 = make_double2(phi0.x + a * (psi1.x + psi0.x), phi0.y + a * (psi1.y + psi0.y));
    if (zero) { rho1 = z; phi1 = z; psi1 = z; }
    p.rho1[mo + k] = rho1;
    p.phi1[mo + k] = phi1;
    p.psi1[mo + k] = psi1;
    double2 out[7];
    out[0] = zero ? z : cmi(kx, make_double2(0.5 * (phi0.x + phi1.x), 0.5 * (phi0.y + phi1.y)));
    const double s2 = p.dt * p.kap2 * p.sigma2;
    for (int c = 0; c < 3; c++) {
      const int64_t vi = 3 * mo + (int64_t)c * N + k;
      const double2 A0 = p.A[vi], U0 = p.U[vi];
      double2 U1 = make_double2(c1 * U0.x + c2 * A0.x + s2 * jm[c].x * inv,
                                c1 * U0.y + c2 * A0.y + s2 * jm[c].y * inv);
      double2 A1 = make_double2(A0.x + a * (U1.x + U0.x), A0.y + a * (U1.y + U0.y));
      if (zero) { A1 = z; U1 = z; }
      p.A1[vi] = A1;
      p.U1[vi] = U1;
      out[1 + c] = A1;
      out[4 + c] = zero ? z : make_double2(0.5 * (U0.x + U1.x), 0.5 * (U0.y + U1.y));
    }
    for (int c = 0; c < nout; c++) sm[c * N + k] = out[c];
  }
  __syncthreads();
  smem_bitrev(sm, nout, N, logN);
  smem_fft(sm, nout, N, p.tw, 1);
  const double in_n = 1.0 / N;
  for (int g = threadIdx.x; g < N; g += blockDim.x) {
    T *rec = nodes + (mo + g) * 8;
    const double gphi = sm[g].x * in_n;
    rec[0] = (T)gphi;
    for (int c = 0; c < 3; c++) {
      const int64_t vi = 3 * mo + (int64_t)c * N + g;
      const double a1 = sm[(1 + c) * N + g].x * in_n;
      rec[1 + c] = (T)p.A_real[vi];
      rec[4 + c] = (T)a1;
      p.A1_real[vi] = a1;
    }
    rec[7] = (T)0;
    if (mode == B_FINAL) {
      for (int c = 0; c < 3; c++) {
        const double uh = sm[(4 + c) * N + g].x * in_n;
        nodes_u[(mo + g) * 4 + c] = (T)uh;
        p.Eh[3 * mo + (int64_t)c * N + g] = -uh - (c == 0 ? gphi : 0.0);
      }
      nodes_u[(mo + g) * 4 + 3] = (T)0;
    }
  }
}

// the particle map of all instances in one mode (map_device.cuh); GEN
// selects the general kernel (degree-one shapes, refinement)
template <typename T, bool FIN, bool GEN>
__global__ void __launch_bounds__(kPT, sizeof(T) == 4 ? 4 : 1)
k_bmap(PView<T> pv, const int32_t *__restrict__ blk2inst, const BInst *__restrict__ inst,
       const PGeom *__restrict__ pgs, const T *__restrict__ invdx, KConst<T> kc,
       const T *__restrict__ nodes, const T *__restrict__ nodes_u, double *__restrict__ Jorb,
       EvalCounters *__restrict__ cnt, double *__restrict__ psum,
       const int32_t *__restrict__ work, const BLoop *__restrict__ loop, int nblocks) {
  // a persistent grid walks this round's list of blocks (k_bctl): blocks of
  // instances that do not evaluate in this mode cost nothing
  const int nw = loop->nwork[FIN ? 1 : 0];
  const int32_t *list = work + (FIN ? nblocks : 0);
  for (int w = blockIdx.x; w < nw; w += gridDim.x) {
    __syncthreads();  // the shared scratch of the previous block is free
    const int blk = list[w];
    const int b = blk2inst[blk];
    const BInst in = inst[b];
    PView<T> v = pv;
    v.np = in.pend;
    const MapScale<T> ms = {{invdx[2 * b], T(1), T(1)}, invdx[2 * b + 1]};
    const PGeom pg = pgs[b];
    map_block<1, T, FIN, GEN>(v, blk * (int64_t)kPT + threadIdx.x, nodes + in.moff * 8,
                              nodes_u + in.moff * 4, Jorb + 3 * in.moff, pg, kc, ms, cnt + b,
                              psum + 2 * (size_t)blk);
  }
}

// H = P J_orb (the real-space Nyquist projector: in 1D, subtract the
// alternating mean times (-1)^g), r_t = H - j_t, the outer-test sums, the
// Gram products of the listed history columns and r_t, and on the final pass
// the particle and mesh work sums (Eq. work-diagnostic) and the chain sum.
__global__ void __launch_bounds__(kBT) k_bresid(BMesh p, double tau_r, double tau_a, int project) {
  __shared__ double sh[kBT / 32];
  __shared__ CSum shc[kBT / 32];
  __shared__ double s_nyq[3];
  __shared__ double s_dots[kNDots];
  const int b = blockIdx.x;
  const BState &s = p.st[b];
  const int mode = s.mode;
  if (mode == B_IDLE) return;
  const BInst in = p.inst[b];
  const int N = in.nx;
  const int64_t base = 3 * in.moff;
  for (int c = 0; c < 3; c++) {
    double v = 0.0;
    for (int g = threadIdx.x; g < N; g += blockDim.x) {
      const double x = p.Jorb[base + c * N + g];
      v += (g & 1) ? -x : x;
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0) s_nyq[c] = project ? v / N : 0.0;
  }
  __syncthreads();
  // the outer tests' norms and the mesh work sum: compensated
  CSum r2 = csum_zero(), h2 = csum_zero(), j2 = csum_zero(), work = csum_zero();
  double mx = 0.0;
  for (int g = threadIdx.x; g < N; g += blockDim.x) {
    double rr = 0.0, hh = 0.0, jj = 0.0;
    for (int c = 0; c < 3; c++) {
      const int64_t q = base + c * N + g;
      const double hv = p.Jorb[q] - ((g & 1) ? -s_nyq[c] : s_nyq[c]);
      const double jv = p.jt[q], rv = hv - jv;
      p.Ht[q] = hv;
      p.rt[q] = rv;
      rr += rv * rv;
      hh += hv * hv;
      jj += jv * jv;
      if (mode == B_FINAL) csum_add(work, hv * p.Eh[q]);
    }
    csum_add(r2, rr);
    csum_add(h2, hh);
    csum_add(j2, jj);
    mx = fmax(mx, sqrt(rr) / (tau_a + 0.5 * tau_r * (sqrt(hh) + sqrt(jj))));
  }
  r2 = block_csum(r2, shc);
  h2 = block_csum(h2, shc);
  j2 = block_csum(j2, shc);
  mx = block_max(mx, sh);
  work = block_csum(work, shc);
  BRes *R = p.res + b;
  if (threadIdx.x == 0) {
    R->r2 = csum_value(r2);
    R->h2 = csum_value(h2);
    R->j2 = csum_value(j2);
    R->smax = mx;
    R->work_mesh = csum_value(work) * in.dx;
  }
  __syncthreads();  // every r_t written
  // Gram products: the warps take the pairs in turn
  const int nc = s.ncol;
  const int npairs = (nc + 1) * (nc + 2) / 2;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int d = wid; d < npairs; d += nw) {
    int a = 0, rem = d;
    while (rem >= nc + 1 - a) {
      rem -= nc + 1 - a;
      a++;
    }
    const int c = a + rem;
    const int sa = a < nc ? s.col[a] : -2, sc = c < nc ? s.col[c] : -2;
    double v = 0.0;
    for (int e = lane; e < 3 * N; e += 32) {
      const int64_t q = base + e;
      const double ra = p.rt[q];
      const double xa = sa >= 0 ? p.dR[sa * p.M3 + q] : (sa == -1 ? ra - p.r[q] : ra);
      const double xc = sc >= 0 ? p.dR[sc * p.M3 + q] : (sc == -1 ? ra - p.r[q] : ra);
      v += xa * xc;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) s_dots[d] = v;
  }
  // final pass: particle work and chain sums of the instance's blocks
  CSum wp = csum_zero(), ch = csum_zero();
  if (mode == B_FINAL)
    for (int k = threadIdx.x; k < in.nblk; k += blockDim.x) {
      csum_add(wp, p.psum[2 * (int64_t)(in.blk0 + k)]);
      csum_add(ch, p.psum[2 * (int64_t)(in.blk0 + k) + 1]);
    }
  wp = block_csum(wp, shc);  // its barriers also publish s_dots
  ch = block_csum(ch, shc);
  if (threadIdx.x == 0) {
    R->work_p = csum_value(wp);
    R->chain = csum_value(ch);
  }
  for (int d = threadIdx.x; d < npairs; d += blockDim.x) R->dots[d] = s_dots[d];
}

// ---- particle kernels over all instances ---------------------------------------

// p^n = P^n - q A^n_h(x^n), A^- and the starting orbit velocity v(p^n)
template <typename T>
__global__ void k_bstep_start(PView<T> pv, T *Am, T *v0, T *vbar,
                              const int32_t *__restrict__ blk2inst,
                              const BInst *__restrict__ inst, const PGeom *__restrict__ pgs,
                              const T *__restrict__ AT, KConst<T> kc) {
  const int b = blk2inst[blockIdx.x];
  const BInst in = inst[b];
  const int64_t i = blockIdx.x * (int64_t)kPT + threadIdx.x;
  if (i >= in.pend) return;
  const PGeom pg = pgs[b];
  int cell[3] = {pv.cell[i], 0, 0};
  T off[3] = {pv.off[i], T(0), T(0)};
  T Ax[3];
  point_interp_T<1, T>(pg, cell, off, AT + 3 * in.moff, Ax);
  const int s = pv.sp[i];
  const T q = (T)(pv.w[i] * kc.qs[s]), m = (T)(pv.w[i] * kc.ms[s]);
  T pp[3], p2 = T(0);
  for (int c = 0; c < 3; c++) {
    Am[c * pv.cap + i] = Ax[c];
    pp[c] = pv.P[c * pv.cap + i] - q * Ax[c];
    p2 += pp[c] * pp[c];
  }
  const T im = T(1) / m, ik = T(1) / kc.kappa;
  const T ig = rsqrt(T(1) + p2 * im * im * ik * ik);
  for (int c = 0; c < 3; c++) {
    const T v = pp[c] * im * ig;
    v0[c * pv.cap + i] = v;
    vbar[c * pv.cap + i] = v;
  }
}

// committed instances: x^{n+1} = x^n + dt vbar, P^{n+1}
template <typename T>
__global__ void k_bcommit(int64_t cap, int32_t *cell, T *off, T *P, const T *__restrict__ vbar,
                          const T *__restrict__ Pnew, const int32_t *__restrict__ blk2inst,
                          const BInst *__restrict__ inst, const BState *__restrict__ st,
                          const T *__restrict__ invdx, double dt) {
  const int b = blk2inst[blockIdx.x];
  if (st[b].phase != B_DONE) return;
  const BInst in = inst[b];
  const int64_t i = blockIdx.x * (int64_t)kPT + threadIdx.x;
  if (i >= in.pend) return;
  const T u = off[i] + (T)dt * vbar[i] * invdx[2 * b];
  const T shf = floor(u + T(0.5));
  cell[i] = (cell[i] + (int)shf) & (in.nx - 1);
  off[i] = u - shf;
  for (int c = 0; c < 3; c++) P[c * cap + i] = Pnew[c * cap + i];
}

// committed instances: n+1 -> n on the mesh, and J_acc <- j
template <typename T>
__global__ void __launch_bounds__(kBT)
k_bcommit_fields(const BInst *__restrict__ inst, const BState *__restrict__ st, double2 *phi,
                 const double2 *phi1, double2 *psi, const double2 *psi1, double2 *rho,
                 const double2 *rho1, double2 *A, const double2 *A1, double2 *U, const double2 *U1,
                 double *A_real, const double *A1_real, T *AT, double *J_acc, const double *j) {
  const int b = blockIdx.x;
  if (st[b].phase != B_DONE) return;
  const BInst in = inst[b];
  const int N = in.nx;
  for (int g = threadIdx.x; g < N; g += blockDim.x) {
    phi[in.moff + g] = phi1[in.moff + g];
    psi[in.moff + g] = psi1[in.moff + g];
    rho[in.moff + g] = rho1[in.moff + g];
  }
  for (int e = threadIdx.x; e < 3 * N; e += blockDim.x) {
    const int64_t q = 3 * in.moff + e;
    A[q] = A1[q];
    U[q] = U1[q];
    A_real[q] = A1_real[q];
    if ((void *)AT != (void *)A_real) AT[q] = (T)A1_real[q];
    J_acc[q] = j[q];
  }
}

// kinetic energy block partials, as in the single-problem context
template <typename T>
__global__ void __launch_bounds__(kPT)
k_bkinetic(PView<T> pv, const int32_t *__restrict__ blk2inst, const BInst *__restrict__ inst,
           const PGeom *__restrict__ pgs, const T *__restrict__ AT, KConst<T> kc, double *psum) {
  const int b = blk2inst[blockIdx.x];
  const BInst in = inst[b];
  const int64_t i = blockIdx.x * (int64_t)kPT + threadIdx.x;
  T k = T(0);
  if (i < in.pend) {
    const PGeom pg = pgs[b];
    int cell[3] = {pv.cell[i], 0, 0};
    T off[3] = {pv.off[i], T(0), T(0)};
    T Ax[3];
    point_interp_T<1, T>(pg, cell, off, AT + 3 * in.moff, Ax);
    const int s = pv.sp[i];
    const T q = (T)(pv.w[i] * kc.qs[s]), m = (T)(pv.w[i] * kc.ms[s]);
    T p2 = T(0);
    for (int c = 0; c < 3; c++) {
      const T pp = pv.P[c * pv.cap + i] - q * Ax[c];
      p2 += pp * pp;
    }
    const T im = T(1) / m;
    const T gam = sqrt(T(1) + p2 * im * im / (kc.kappa * kc.kappa));
    k = p2 * im / (gam + T(1));
  }
  // a warp sums its 32 positive terms plainly; the warps merge with TwoSum
  // into the block's (sum, error) pair
  for (int o = 16; o > 0; o >>= 1) k += __shfl_down_sync(0xffffffffu, k, o);
  __shared__ double sh[kPT / 32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = widen(k);
  __syncthreads();
  if (threadIdx.x == 0) {
    CSum t = csum_zero();
    for (int w = 0; w < kPT / 32; w++) csum_add(t, sh[w]);
    psum[2 * (int64_t)blockIdx.x] = t.s;
    psum[2 * (int64_t)blockIdx.x + 1] = t.c;
  }
}

// per-instance diagnostics: K (from the block partials), the field energy
// (Eq. field-energy-section2) and the Gauss and Lorenz residuals (Eq.
// constraint-residuals), by Parseval as in the single-problem context
__global__ void __launch_bounds__(kBT)
k_bdiag(const BInst *__restrict__ inst, const double *__restrict__ psum, const double2 *phi,
        const double2 *psi, const double2 *rho, const double2 *A, const double2 *U,
        double sigma1, double sigma2, double kap2, double *out) {
  __shared__ CSum shc[kBT / 32];
  const int b = blockIdx.x;
  const BInst in = inst[b];
  const int N = in.nx;
  const double twopiL = 2.0 * M_PI / in.L;
  // every sum compensated, as in the single-problem context
  CSum K = csum_zero();
  for (int k = threadIdx.x; k < in.nblk; k += blockDim.x)
    K = csum_merge(K, CSum{psum[2 * (int64_t)(in.blk0 + k)],
                           psum[2 * (int64_t)(in.blk0 + k) + 1]});
  CSum w = csum_zero(), gs = csum_zero(), ls = csum_zero();
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const bool nyq = k == N / 2;
    const int kk = k < N / 2 ? k : k - N;
    const double kx = nyq ? 0.0 : twopiL * kk;
    const double2 ph = phi[in.moff + k];
    double2 Ah[3], Uh[3];
    for (int c = 0; c < 3; c++) {
      Ah[c] = A[3 * in.moff + (int64_t)c * N + k];
      Uh[c] = U[3 * in.moff + (int64_t)c * N + k];
    }
    double e2 = 0.0;
    for (int c = 0; c < 3; c++) {
      double2 E = make_double2(-Uh[c].x, -Uh[c].y);
      if (c == 0) {  // - i k phi
        E.x += kx * ph.y;
        E.y -= kx * ph.x;
      }
      e2 += E.x * E.x + E.y * E.y;
    }
    // B = curl A with d/dy = d/dz = 0: (0, -i k A_z, i k A_y)
    const double b2 = kx * kx * (Ah[1].x * Ah[1].x + Ah[1].y * Ah[1].y +
                                 Ah[2].x * Ah[2].x + Ah[2].y * Ah[2].y);
    csum_add(w, e2 / (2.0 * sigma1) + b2 / (2.0 * sigma2));
    const double2 rr = rho[in.moff + k], ps = psi[in.moff + k];
    const double2 divU = cmi(kx, Uh[0]), divA = cmi(kx, Ah[0]);
    const double RGx = kx * kx * ph.x - divU.x - sigma1 * rr.x;
    const double RGy = kx * kx * ph.y - divU.y - sigma1 * rr.y;
    const double RLx = ps.x / kap2 + divA.x, RLy = ps.y / kap2 + divA.y;
    csum_add(gs, RGx * RGx + RGy * RGy);
    csum_add(ls, RLx * RLx + RLy * RLy);
  }
  K = block_csum(K, shc);
  w = block_csum(w, shc);
  gs = block_csum(gs, shc);
  ls = block_csum(ls, shc);
  if (threadIdx.x == 0) {
    out[4 * b] = csum_value(K);
    out[4 * b + 1] = csum_value(w) * in.dx / N;
    out[4 * b + 2] = sqrt(csum_value(gs)) / N;
    out[4 * b + 3] = sqrt(csum_value(ls)) / N;
  }
}

// accepted particles of one instance in load order: x, P, w, species
template <typename T>
__global__ void k_bexport(int64_t cap, const int32_t *__restrict__ cell, const T *__restrict__ off,
                          const T *__restrict__ P, const double *__restrict__ w,
                          const int32_t *__restrict__ sp, const int64_t *__restrict__ id,
                          BInst in, double *x_out, double *P_out, double *w_out, int32_t *sp_out) {
  const int64_t i = in.pbeg + blockIdx.x * (int64_t)kPT + threadIdx.x;
  if (i >= in.pend) return;
  const int64_t n = in.pend - in.pbeg, j = id[i];
  double u = (double)cell[i] + (double)off[i];
  if (u < 0.0) u += (double)in.nx;
  x_out[j] = in.x0 + u * in.dx;
  for (int c = 0; c < 3; c++) P_out[c * n + j] = (double)P[c * cap + i];
  w_out[j] = w[i];
  sp_out[j] = sp[i];
}

// the accepted potentials of one instance in real space: phi, psi, rho, A, U
__global__ void __launch_bounds__(kBT)
k_bto_real(BInst in, const double2 *phi, const double2 *psi, const double2 *rho, const double2 *A,
           const double2 *U, const double2 *tw, double *out) {
  extern __shared__ double2 sm[];
  const int N = in.nx;
  for (int t = threadIdx.x; t < 9 * N; t += blockDim.x) {
    const int c = t / N, g = t - c * N;
    double2 v;
    if (c == 0) v = phi[in.moff + g];
    else if (c == 1) v = psi[in.moff + g];
    else if (c == 2) v = rho[in.moff + g];
    else if (c < 6) v = A[3 * in.moff + (int64_t)(c - 3) * N + g];
    else v = U[3 * in.moff + (int64_t)(c - 6) * N + g];
    sm[c * N + brev(g, in.logn)] = v;
  }
  __syncthreads();
  smem_fft(sm, 9, N, tw, 1);
  for (int t = threadIdx.x; t < 9 * N; t += blockDim.x) out[t] = sm[t].x / N;
}

// ---- segmented counting sort by cell (every instance keeps its range) ----------
__global__ void k_bsort_keys(const int32_t *__restrict__ blk2inst, const BInst *__restrict__ inst,
                             const int32_t *__restrict__ cell, int32_t *keys, int32_t *count) {
  const int b = blk2inst[blockIdx.x];
  const BInst in = inst[b];
  const int64_t i = blockIdx.x * (int64_t)kPT + threadIdx.x;
  if (i >= in.pend) return;
  const int k = (int)in.moff + cell[i];
  keys[i] = k;
  atomicAdd(count + k, 1);
}

// exclusive scan of count[0, n) in place (one block of 1024 threads)
__global__ void k_bsort_scan(int32_t *count, int n) {
  __shared__ int32_t sh[1024];
  const int chunk = (n + 1023) / 1024;
  const int t0 = threadIdx.x * chunk;
  int32_t s = 0;
  for (int k = t0; k < min(t0 + chunk, n); k++) s += count[k];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int32_t v = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  int32_t run = sh[threadIdx.x] - s;
  for (int k = t0; k < min(t0 + chunk, n); k++) {
    const int32_t c = count[k];
    count[k] = run;
    run += c;
  }
}

__global__ void k_bsort_slots(const int32_t *__restrict__ blk2inst, const BInst *__restrict__ inst,
                              const int32_t *__restrict__ keys, int32_t *cursor, int64_t *slot) {
  const int b = blk2inst[blockIdx.x];
  const BInst in = inst[b];
  const int64_t i = blockIdx.x * (int64_t)kPT + threadIdx.x;
  if (i >= in.pend) return;
  slot[i] = (int64_t)atomicAdd(cursor + keys[i], 1) + in.sort_shift;
}

template <typename V>
__global__ void k_bpermute(const int32_t *__restrict__ blk2inst, const BInst *__restrict__ inst,
                           int64_t cap, int ncomp, const V *__restrict__ src, V *__restrict__ dst,
                           const int64_t *__restrict__ slot) {
  const int b = blk2inst[blockIdx.x];
  const BInst in = inst[b];
  const int64_t i = blockIdx.x * (int64_t)kPT + threadIdx.x;
  if (i >= in.pend) return;
  const int64_t j = slot[i];
  for (int c = 0; c < ncomp; c++) dst[c * cap + j] = src[c * cap + i];
}

// ---- host side -----------------------------------------------------------------

bool b_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int b_log2(int n) {
  int l = 0;
  while ((1 << l) < n) l++;
  return l;
}

// effective tolerances, as the single-problem context (mixed floor, reading R9)
void b_tolerances(const pic_batch *bt, double tol, double *tr, double *ta, double *itr,
                  double *ita) {
  double t = tol;
  if (bt->opt.precision == PIC_MIXED) t = std::max(t, bt->opt.mixed_tol_floor);
  *tr = t;
  *ta = t * bt->opt.tol_abs_ratio;
  double ti = tol * bt->opt.inner_tol_scale;
  if (bt->opt.precision == PIC_MIXED) ti = std::max(ti, bt->opt.mixed_tol_floor);
  *itr = ti;
  *ita = ti * bt->opt.tol_abs_ratio;
}

template <typename T>
KConst<T> b_kconst(const pic_batch *bt, double itr, double ita) {
  StepConst sc;
  std::memset(&sc, 0, sizeof sc);
  sc.dt = bt->dt;
  sc.kappa = bt->opt.kappa;
  for (int s = 0; s < PIC_MAX_SPECIES; s++) {
    sc.qs[s] = s < bt->nspecies ? bt->qs[s] : 0.0;
    sc.ms[s] = s < bt->nspecies ? bt->ms[s] : 1.0;
  }
  sc.tau_r = itr;
  sc.tau_a = ita;
  sc.inner_max = bt->opt.inner_max;
  sc.ngl = bt->opt.gl_points > 0 ? bt->opt.gl_points : 2;  // minimal exact count in 1D
  sc.warm = bt->opt.inner_warm_start ? 1 : 0;
  sc.order = bt->opt.order;
  sc.refine_max = bt->opt.refine_max;
  gauss_legendre01(sc.ngl, sc.gl_t, sc.gl_w);
  PGeom unit;
  std::memset(&unit, 0, sizeof unit);
  for (int l = 0; l < 3; l++) unit.inv_dx[l] = 1.0;
  unit.inv_dV = 1.0;  // per-instance values are set by the kernels
  return kconst<T>(sc, unit);
}

template <typename T>
PView<T> b_pview(const pic_batch *bt) {
  PView<T> v;
  v.np = 0;
  v.cap = bt->cap;
  v.cell = bt->cell;
  v.off = (const T *)bt->off;
  v.P = (const T *)bt->P;
  v.Am = (const T *)bt->Am;
  v.v0 = (const T *)bt->v0;
  v.w = bt->w;
  v.sp = bt->sp;
  v.vbar = (T *)bt->vbar;
  v.Pnew = (T *)bt->Pnew;
  v.iters = bt->iters;
  return v;
}

BMesh b_mesh(const pic_batch *bt) {
  BMesh m;
  m.inst = bt->d_inst;
  m.st = bt->d_state;
  m.j = bt->j;
  m.jt = bt->jt;
  m.H = bt->H;
  m.Ht = bt->Ht;
  m.r = bt->r;
  m.rt = bt->rt;
  m.dJ = bt->dJ;
  m.dR = bt->dR;
  m.Jorb = bt->Jorb;
  m.Eh = bt->Eh;
  m.J_acc = bt->J_acc;
  m.M3 = 3 * bt->M;
  m.res = bt->d_res;
  m.cnt = bt->d_cnt;
  m.psum = bt->psum;
  return m;
}

BParams b_params(const pic_batch *bt, double tr, double ta) {
  BParams bp;
  bp.M = bt->opt.anderson_m;
  bp.anderson_start = bt->opt.anderson_start;
  bp.levels = bt->opt.backtrack_levels;
  bp.outer_max = bt->opt.outer_max;
  bp.beta = bt->opt.beta;
  bp.lambda = bt->opt.lambda;
  bp.dc = bt->opt.decrease_coef;
  bp.growth = bt->opt.growth_limit;
  bp.growth_scaled = bt->opt.growth_scaled;
  bp.tr = tr;
  bp.ta = ta;
  return bp;
}

size_t field_smem(const pic_batch *bt) {
  int nmax = 4;
  for (const BInst &in : bt->inst) nmax = std::max(nmax, in.nx);
  return sizeof(double2) * 9 * (size_t)nmax;  // 7 lines for k_bfield, 9 for k_bto_real
}

// the kernels of one round (see the file comment)
// persistent grid of a particle-map variant: every SM filled with as many
// CTAs as it holds, never more CTAs than blocks
template <typename T, bool FIN, bool GEN>
int map_grid(pic_batch *bt) {
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bmap<T, FIN, GEN>, kPT, 0) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return std::max(1, std::min(bt->nblocks, per_sm * bt->num_sms));
}

// rounds a step may take: every round is one evaluation per running
// instance, Algorithm 1 needs at most 2 + outer_max (2 levels + 1) of them,
// and one more round finds no instance running
int max_rounds(const pic_batch *bt) {
  return 4 + bt->opt.outer_max * (2 * bt->opt.backtrack_levels + 1);
}

template <typename T>
int enqueue_round(pic_batch *bt, double tr, double ta, double itr, double ita,
                  cudaGraphConditionalHandle cond) {
  const int B = bt->B;
  const BMesh m = b_mesh(bt);
  k_bctl<<<1, kCtlThreads, 0, bt->st>>>(B, bt->d_state, bt->d_res, bt->d_cnt, bt->d_inst,
                                         b_params(bt, tr, ta), bt->d_loop, max_rounds(bt), cond,
                                         bt->d_work, bt->nblocks);
  BKCHECK();
  k_baccept<<<B, kBT, 0, bt->st>>>(m);
  BKCHECK();
  k_btrial<<<B, kBT, 0, bt->st>>>(m);
  BKCHECK();
  BField f;
  f.inst = bt->d_inst;
  f.st = bt->d_state;
  f.jt = bt->jt;
  f.A_real = bt->A_real;
  f.rho = bt->rho_h;
  f.phi = bt->phi_h;
  f.psi = bt->psi_h;
  f.A = bt->A_h;
  f.U = bt->U_h;
  f.rho1 = bt->rho1_h;
  f.phi1 = bt->phi1_h;
  f.psi1 = bt->psi1_h;
  f.A1 = bt->A1_h;
  f.U1 = bt->U1_h;
  f.A1_real = bt->A1_real;
  f.Jorb = bt->Jorb;
  f.Eh = bt->Eh;
  f.tw = bt->tw;
  f.dt = bt->dt;
  f.kap2 = bt->opt.kappa * bt->opt.kappa;
  f.sigma1 = bt->opt.sigma1;
  f.sigma2 = bt->opt.sigma2;
  f.project = bt->opt.project_nyquist;
  k_bfield<T><<<B, kBT, field_smem(bt), bt->st>>>(f, (T *)bt->nodes, (T *)bt->nodes_u);
  BKCHECK();
  if (bt->nblocks > 0) {
    const KConst<T> kc = b_kconst<T>(bt, itr, ita);
#define B_MAP_LAUNCH(FIN, GEN)                                                                \
  k_bmap<T, FIN, GEN><<<map_grid<T, FIN, GEN>(bt), kPT, 0, bt->st>>>(                         \
      b_pview<T>(bt), bt->d_blk2inst, bt->d_inst, bt->d_pg, (const T *)bt->d_invdx, kc,         \
      (const T *)bt->nodes, (const T *)bt->nodes_u, bt->Jorb, bt->d_cnt, bt->psum, bt->d_work,  \
      bt->d_loop, bt->nblocks)
    if (bt->opt.order != 2 || bt->opt.refine_max > 0) {
      B_MAP_LAUNCH(false, true);
      BKCHECK();
      B_MAP_LAUNCH(true, true);
    } else {
      B_MAP_LAUNCH(false, false);
      BKCHECK();
      B_MAP_LAUNCH(true, false);
    }
#undef B_MAP_LAUNCH
    BKCHECK();
    bt->map_launches += 2;
  }
  k_bresid<<<B, kBT, 0, bt->st>>>(m, tr, ta, bt->opt.project_nyquist);
  BKCHECK();
  return PIC_OK;
}

// Build the graph of a step's round loop: one conditional while node whose
// body is the round, captured from the same launches the host-driven
// fallback makes; k_bctl sets the node's condition.  Returns false (and
// leaves no error pending) if the driver cannot build it.
bool build_loop_graph(pic_batch *bt, double tr, double ta, double itr, double ita) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
  cudaGraphConditionalHandle cond = 0;
  if (ok) ok = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) ==
               cudaSuccess;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node = nullptr;
  if (ok) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
  }
  if (ok) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(bt->st, body, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const long long before = bt->launches, mbefore = bt->map_launches;
      const int e = bt->rsize == 8 ? enqueue_round<double>(bt, tr, ta, itr, ita, cond)
                                   : enqueue_round<float>(bt, tr, ta, itr, ita, cond);
      bt->launches = before;
      bt->map_launches = mbefore;
      cudaGraph_t cap = nullptr;
      ok = cudaStreamEndCapture(bt->st, &cap) == cudaSuccess && e == PIC_OK;
    }
  }
  if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();  // a refused build falls back to host-driven rounds
  if (!ok) {
    if (exec) cudaGraphExecDestroy(exec);
    return false;
  }
  if (bt->loop_exec) cudaGraphExecDestroy(bt->loop_exec);
  bt->loop_exec = exec;
  bt->graph_tr = tr;
  bt->graph_ta = ta;
  bt->graph_itr = itr;
  bt->graph_ita = ita;
  return true;
}

// Queue all rounds of a step.  With the loop graph, one graph launch runs
// them with no host round trip; otherwise the host launches a round, reads
// the loop state and repeats.
int b_rounds(pic_batch *bt, double tr, double ta, double itr, double ita) {
  if (bt->graph_ok == 1 && (bt->graph_tr != tr || bt->graph_ta != ta || bt->graph_itr != itr ||
                            bt->graph_ita != ita))
    bt->graph_ok = 0;
  if (bt->graph_ok == 0)
    bt->graph_ok = !bt->opt.host_control && build_loop_graph(bt, tr, ta, itr, ita) ? 1 : -1;
  if (bt->graph_ok == 1) {
    BCK(cudaGraphLaunch(bt->loop_exec, bt->st));
    return PIC_OK;  // launches are counted from the rounds the loop reports
  }
  for (;;) {
    const int e = bt->rsize == 8 ? enqueue_round<double>(bt, tr, ta, itr, ita, 0)
                                 : enqueue_round<float>(bt, tr, ta, itr, ita, 0);
    if (e) return e;
    BCK(cudaMemcpyAsync(bt->h_loop, bt->d_loop, sizeof(BLoop), cudaMemcpyDeviceToHost, bt->st));
    BCK(cudaStreamSynchronize(bt->st));
    if (bt->h_loop->running == 0 || bt->h_loop->overflow) return PIC_OK;
  }
}

template <typename T>
int b_step_start(pic_batch *bt) {
  const int B = bt->B;
  k_bbegin<<<(B + 255) / 256, 256, 0, bt->st>>>(B, bt->d_state, bt->d_loop);
  BKCHECK();
  if (bt->nblocks > 0) {
    k_bstep_start<T><<<bt->nblocks, kPT, 0, bt->st>>>(
        b_pview<T>(bt), (T *)bt->Am, (T *)bt->v0, (T *)bt->vbar, bt->d_blk2inst, bt->d_inst,
        bt->d_pg, (const T *)bt->AT, b_kconst<T>(bt, 0.0, 0.0));
    BKCHECK();
  }
  return PIC_OK;
}

// commit the finished instances, then the diagnostics of every instance
template <typename T>
int b_commit_diag(pic_batch *bt) {
  const int B = bt->B;
  if (bt->nblocks > 0) {
    k_bcommit<T><<<bt->nblocks, kPT, 0, bt->st>>>(bt->cap, bt->cell, (T *)bt->off, (T *)bt->P,
                                                  (const T *)bt->vbar, (const T *)bt->Pnew,
                                                  bt->d_blk2inst, bt->d_inst, bt->d_state,
                                                  (const T *)bt->d_invdx, bt->dt);
    BKCHECK();
  }
  k_bcommit_fields<T><<<B, kBT, 0, bt->st>>>(bt->d_inst, bt->d_state, bt->phi_h, bt->phi1_h,
                                             bt->psi_h, bt->psi1_h, bt->rho_h, bt->rho1_h,
                                             bt->A_h, bt->A1_h, bt->U_h, bt->U1_h, bt->A_real,
                                             bt->A1_real, (T *)bt->AT, bt->J_acc, bt->j);
  BKCHECK();
  return PIC_OK;
}

template <typename T>
int b_diag(pic_batch *bt) {
  if (bt->nblocks > 0) {
    k_bkinetic<T><<<bt->nblocks, kPT, 0, bt->st>>>(b_pview<T>(bt), bt->d_blk2inst, bt->d_inst,
                                                   bt->d_pg, (const T *)bt->AT,
                                                   b_kconst<T>(bt, 0.0, 0.0), bt->psum);
    BKCHECK();
  }
  k_bdiag<<<bt->B, kBT, 0, bt->st>>>(bt->d_inst, bt->psum, bt->phi_h, bt->psi_h, bt->rho_h,
                                     bt->A_h, bt->U_h, bt->opt.sigma1, bt->opt.sigma2,
                                     bt->opt.kappa * bt->opt.kappa, bt->d_diag);
  BKCHECK();
  BCK(cudaMemcpyAsync(bt->h_diag, bt->d_diag, sizeof(double) * 4 * bt->B, cudaMemcpyDeviceToHost,
                      bt->st));
  return PIC_OK;
}

template <typename V>
int b_permute(pic_batch *bt, V *field, int ncomp) {
  V *scr = (V *)bt->tmp_r;  // 3 * cap * 8 bytes of scratch
  k_bpermute<V><<<bt->nblocks, kPT, 0, bt->st>>>(bt->d_blk2inst, bt->d_inst, bt->cap, ncomp, field,
                                                 scr, bt->slot);
  BKCHECK();
  BCK(cudaMemcpyAsync(field, scr, sizeof(V) * ncomp * bt->cap, cudaMemcpyDeviceToDevice, bt->st));
  return PIC_OK;
}

int b_sort(pic_batch *bt) {
  if (bt->nblocks == 0) return PIC_OK;
  BCK(cudaMemsetAsync(bt->cnt_sort, 0, sizeof(int32_t) * bt->M, bt->st));
  k_bsort_keys<<<bt->nblocks, kPT, 0, bt->st>>>(bt->d_blk2inst, bt->d_inst, bt->cell, bt->keys,
                                                bt->cnt_sort);
  BKCHECK();
  k_bsort_scan<<<1, 1024, 0, bt->st>>>(bt->cnt_sort, (int)bt->M);
  BKCHECK();
  k_bsort_slots<<<bt->nblocks, kPT, 0, bt->st>>>(bt->d_blk2inst, bt->d_inst, bt->keys,
                                                 bt->cnt_sort, bt->slot);
  BKCHECK();
  int e;
  if ((e = b_permute<int32_t>(bt, bt->cell, 1))) return e;
  if ((e = b_permute<int32_t>(bt, bt->sp, 1))) return e;
  if ((e = b_permute<double>(bt, bt->w, 1))) return e;
  if ((e = b_permute<int64_t>(bt, bt->id, 1))) return e;
  if (bt->rsize == 8) {
    if ((e = b_permute<double>(bt, (double *)bt->off, 1))) return e;
    if ((e = b_permute<double>(bt, (double *)bt->P, 3))) return e;
  } else {
    if ((e = b_permute<float>(bt, (float *)bt->off, 1))) return e;
    if ((e = b_permute<float>(bt, (float *)bt->P, 3))) return e;
  }
  return PIC_OK;
}

void b_free_all(pic_batch *bt) {
  if (bt->loop_exec) cudaGraphExecDestroy(bt->loop_exec);
  void *dev[] = {bt->d_inst, bt->d_pg, bt->d_invdx, bt->d_blk2inst, bt->d_work, bt->d_state,
                 bt->d_res, bt->d_cnt, bt->d_loop, bt->cell, bt->sp, bt->iters, bt->keys, bt->cnt_sort,
                 bt->id, bt->slot, bt->off, bt->P, bt->Am, bt->v0, bt->vbar, bt->Pnew, bt->tmp_r,
                 bt->w, bt->psum, bt->phi_h, bt->psi_h, bt->rho_h, bt->A_h, bt->U_h, bt->phi1_h,
                 bt->psi1_h, bt->rho1_h, bt->A1_h, bt->U1_h, bt->A_real, bt->A1_real, bt->J_acc,
                 bt->Jorb, bt->j, bt->jt, bt->H, bt->Ht, bt->r, bt->rt, bt->Eh, bt->dJ, bt->dR,
                 bt->nodes, bt->nodes_u, bt->tw, bt->d_diag, bt->d_out};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (bt->AT && bt->AT != (void *)bt->A_real) cudaFree(bt->AT);
  if (bt->h_state) cudaFreeHost(bt->h_state);
  if (bt->h_loop) cudaFreeHost(bt->h_loop);
  if (bt->h_diag) cudaFreeHost(bt->h_diag);
  if (bt->own_st) cudaStreamDestroy(bt->own_st);
}

const char *why_text(int why) {
  switch (why) {
    case W_INNER: return "inner particle solve failed";
    case W_LIMIT: return "outer iteration limit reached";
    case W_NODIR: return "no accepted outer direction";
    case W_VERIFY: return "verification evaluation failed the outer tests";
    default: return "";
  }
}

}  // namespace

extern "C" {

int pic_batch_init(pic_batch **out, int B, const int *n, const double *L, const double *x0,
                   const int64_t *np, const pic_species *species, int nspecies, double dt,
                   const pic_options *opt) {
  if (!out) return PIC_EARG;
  *out = nullptr;
  if (B < 1 || B > 65536 || !n || !L || !np || !species || nspecies < 1 ||
      nspecies > PIC_MAX_SPECIES || !(dt > 0.0))
    return PIC_EARG;
  pic_options o;
  if (opt) o = *opt;
  else pic_default_options(&o);
  if (o.anderson_m < 0 || o.anderson_m > kMh || o.backtrack_levels < 1 || o.outer_max < 1 ||
      o.inner_max < 1 || o.gl_points < 0 || o.gl_points > PIC_MAX_GL ||
      (o.precision != PIC_FP64 && o.precision != PIC_MIXED) || !(o.kappa > 0.0) ||
      (o.order != 1 && o.order != 2) || o.refine_max < 0 || o.refine_max > 3 ||
      o.deterministic_deposit)  // the batch deposits with atomics only
    return PIC_EARG;
  for (int s = 0; s < nspecies; s++)
    if (!(species[s].m > 0.0)) return PIC_EARG;
  int64_t ntot = 0;
  for (int b = 0; b < B; b++) {
    if (!b_pow2(n[b]) || n[b] < 4 || n[b] > kNmax || !(L[b] > 0.0) || np[b] < 0) return PIC_EARG;
    ntot += np[b];
  }
  if (ntot > ((int64_t)1 << 31) - (int64_t)kPT * B) return PIC_EARG;  // int32 sort cursors
  pic_batch *bt = new pic_batch();
  bt->B = B;
  bt->nspecies = nspecies;
  for (int s = 0; s < PIC_MAX_SPECIES; s++) {
    bt->qs[s] = s < nspecies ? species[s].q : 0.0;
    bt->ms[s] = s < nspecies ? species[s].m : 1.0;
  }
  bt->dt = dt;
  bt->opt = o;
  bt->rsize = o.precision == PIC_MIXED ? 4 : 8;
  bt->st = (cudaStream_t)o.cuda_stream;
  if (!bt->st) {
    if (cudaStreamCreate(&bt->own_st) != cudaSuccess) {
      cudaGetLastError();
      delete bt;
      return PIC_ECUDA;
    }
    bt->st = bt->own_st;
  }
  {
    int dev = 0;
    bt->num_sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&bt->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      cudaGetLastError();
  }
  // instance table: meshes back to back, particle ranges padded to kPT
  bt->inst.resize(B);
  bt->np.assign(np, np + B);
  bt->E0.assign(B, 0.0);
  bt->stage.resize(B);
  int64_t moff = 0, p = 0, before = 0;
  int blk = 0;
  std::vector<int32_t> b2i;
  std::vector<PGeom> pgs(B);
  for (int b = 0; b < B; b++) {
    BInst &in = bt->inst[b];
    in.nx = n[b];
    in.logn = b_log2(n[b]);
    in.moff = moff;
    in.pbeg = p;
    in.pend = p + np[b];
    in.blk0 = blk;
    in.nblk = (int)((np[b] + kPT - 1) / kPT);
    in.sort_shift = p - before;
    in.L = L[b];
    in.x0 = x0 ? x0[b] : 0.0;
    in.dx = L[b] / n[b];
    for (int k = 0; k < in.nblk; k++) b2i.push_back(b);
    moff += n[b];
    p += (int64_t)in.nblk * kPT;
    blk += in.nblk;
    before += np[b];
    PGeom &pg = pgs[b];
    std::memset(&pg, 0, sizeof pg);
    for (int a = 0; a < 3; a++) {
      pg.n[a] = a == 0 ? n[b] : 1;
      pg.mask[a] = pg.n[a] - 1;
      pg.dx[a] = a == 0 ? in.dx : 1.0;
      pg.inv_dx[a] = 1.0 / pg.dx[a];
      pg.x0[a] = a == 0 ? in.x0 : 0.0;
      pg.L[a] = a == 0 ? L[b] : 1.0;
    }
    pg.Ng = n[b];
    pg.n0 = n[b];
    pg.n01 = n[b];
    pg.order = o.order;
    pg.inv_dV = 1.0 / in.dx;
  }
  bt->M = moff;
  bt->cap = std::max<int64_t>(p, 1);
  bt->nblocks = blk;
  const int64_t M = bt->M, cap = bt->cap;
  const size_t R = bt->rsize;
  const int Mh = std::max(o.anderson_m, 1);
  struct Alloc {
    void **p;
    size_t bytes;
  };
  const std::vector<Alloc> allocs = {
      {(void **)&bt->d_inst, sizeof(BInst) * B},
      {(void **)&bt->d_pg, sizeof(PGeom) * B},
      {&bt->d_invdx, R * 2 * B},
      {(void **)&bt->d_blk2inst, sizeof(int32_t) * std::max(blk, 1)},
      {(void **)&bt->d_work, sizeof(int32_t) * 2 * std::max(blk, 1)},
      {(void **)&bt->d_state, sizeof(BState) * B},
      {(void **)&bt->d_res, sizeof(BRes) * B},
      {(void **)&bt->d_cnt, sizeof(EvalCounters) * B},
      {(void **)&bt->d_loop, sizeof(BLoop)},
      {(void **)&bt->cell, sizeof(int32_t) * cap},
      {(void **)&bt->sp, sizeof(int32_t) * cap},
      {(void **)&bt->iters, sizeof(int32_t) * cap},
      {(void **)&bt->keys, sizeof(int32_t) * cap},
      {(void **)&bt->cnt_sort, sizeof(int32_t) * M},
      {(void **)&bt->id, sizeof(int64_t) * cap},
      {(void **)&bt->slot, sizeof(int64_t) * cap},
      {&bt->off, R * cap},
      {&bt->P, R * 3 * cap},
      {&bt->Am, R * 3 * cap},
      {&bt->v0, R * 3 * cap},
      {&bt->vbar, R * 3 * cap},
      {&bt->Pnew, R * 3 * cap},
      {&bt->tmp_r, sizeof(double) * 3 * cap},
      {(void **)&bt->w, sizeof(double) * cap},
      {(void **)&bt->psum, sizeof(double) * 2 * std::max(blk, 1)},
      {(void **)&bt->phi_h, sizeof(double2) * M},
      {(void **)&bt->psi_h, sizeof(double2) * M},
      {(void **)&bt->rho_h, sizeof(double2) * M},
      {(void **)&bt->A_h, sizeof(double2) * 3 * M},
      {(void **)&bt->U_h, sizeof(double2) * 3 * M},
      {(void **)&bt->phi1_h, sizeof(double2) * M},
      {(void **)&bt->psi1_h, sizeof(double2) * M},
      {(void **)&bt->rho1_h, sizeof(double2) * M},
      {(void **)&bt->A1_h, sizeof(double2) * 3 * M},
      {(void **)&bt->U1_h, sizeof(double2) * 3 * M},
      {(void **)&bt->A_real, sizeof(double) * 3 * M},
      {(void **)&bt->A1_real, sizeof(double) * 3 * M},
      {(void **)&bt->J_acc, sizeof(double) * 3 * M},
      {(void **)&bt->Jorb, sizeof(double) * 3 * M},
      {(void **)&bt->j, sizeof(double) * 3 * M},
      {(void **)&bt->jt, sizeof(double) * 3 * M},
      {(void **)&bt->H, sizeof(double) * 3 * M},
      {(void **)&bt->Ht, sizeof(double) * 3 * M},
      {(void **)&bt->r, sizeof(double) * 3 * M},
      {(void **)&bt->rt, sizeof(double) * 3 * M},
      {(void **)&bt->Eh, sizeof(double) * 3 * M},
      {(void **)&bt->dJ, sizeof(double) * 3 * M * Mh},
      {(void **)&bt->dR, sizeof(double) * 3 * M * Mh},
      {&bt->nodes, R * 8 * M},
      {&bt->nodes_u, R * 4 * M},
      {(void **)&bt->tw, sizeof(double2) * kNmax / 2},
      {(void **)&bt->d_diag, sizeof(double) * 4 * B},
      {(void **)&bt->d_out, sizeof(double) * std::max<int64_t>(9 * kNmax, 6 * cap)},
  };
  for (const Alloc &a : allocs) {
    if (cudaMalloc(a.p, a.bytes) != cudaSuccess) {
      cudaGetLastError();
      b_free_all(bt);
      delete bt;
      return PIC_ENOMEM;
    }
  }
  if (bt->rsize == 8) {
    bt->AT = bt->A_real;
  } else if (cudaMalloc(&bt->AT, sizeof(float) * 3 * M) != cudaSuccess) {
    cudaGetLastError();
    b_free_all(bt);
    delete bt;
    return PIC_ENOMEM;
  }
  if (cudaMallocHost((void **)&bt->h_state, sizeof(BState) * B) != cudaSuccess ||
      cudaMallocHost((void **)&bt->h_loop, sizeof(BLoop)) != cudaSuccess ||
      cudaMallocHost((void **)&bt->h_diag, sizeof(double) * 4 * B) != cudaSuccess) {
    cudaGetLastError();
    b_free_all(bt);
    delete bt;
    return PIC_ENOMEM;
  }
  // constant tables
  std::vector<double2> tw(kNmax / 2);
  for (int k = 0; k < kNmax / 2; k++) {
    const double ang = -2.0 * M_PI * k / kNmax;
    tw[k] = make_double2(std::cos(ang), std::sin(ang));
  }
  std::vector<char> invdx(R * 2 * B);
  for (int b = 0; b < B; b++) {
    const double v = 1.0 / bt->inst[b].dx;  // 1/dx and 1/dV coincide in 1D
    for (int q = 0; q < 2; q++) {
      if (R == 8) {
        std::memcpy(&invdx[(2 * b + q) * 8], &v, 8);
      } else {
        const float f = (float)v;
        std::memcpy(&invdx[(2 * b + q) * 4], &f, 4);
      }
    }
  }
  int e = PIC_OK;
  if (cudaMemcpy(bt->d_inst, bt->inst.data(), sizeof(BInst) * B, cudaMemcpyHostToDevice) ||
      cudaMemcpy(bt->d_pg, pgs.data(), sizeof(PGeom) * B, cudaMemcpyHostToDevice) ||
      cudaMemcpy(bt->d_invdx, invdx.data(), invdx.size(), cudaMemcpyHostToDevice) ||
      cudaMemcpy(bt->tw, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice) ||
      (blk > 0 &&
       cudaMemcpy(bt->d_blk2inst, b2i.data(), sizeof(int32_t) * blk, cudaMemcpyHostToDevice)) ||
      cudaMemset(bt->d_res, 0, sizeof(BRes) * B) ||
      cudaMemset(bt->d_cnt, 0, sizeof(EvalCounters) * B) ||
      cudaMemset(bt->d_state, 0, sizeof(BState) * B) ||
      cudaMemset(bt->dJ, 0, sizeof(double) * 3 * M * Mh) ||
      cudaMemset(bt->dR, 0, sizeof(double) * 3 * M * Mh) ||
      cudaMemset(bt->r, 0, sizeof(double) * 3 * M) ||
      cudaMemset(bt->nodes_u, 0, R * 4 * M))
    e = PIC_ECUDA;
  const size_t smem = field_smem(bt);
  if (!e && smem > 48 * 1024) {
    if (cudaFuncSetAttribute(k_bfield<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) ||
        cudaFuncSetAttribute(k_bfield<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) ||
        cudaFuncSetAttribute(k_bto_real, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
      e = PIC_ECUDA;
  }
  if (e) {
    cudaGetLastError();
    b_free_all(bt);
    delete bt;
    return e;
  }
  *out = bt;
  return PIC_OK;
}

void pic_batch_free(pic_batch *bt) {
  if (!bt) return;
  cudaStreamSynchronize(bt->st);
  b_free_all(bt);
  delete bt;
}

const char *pic_batch_last_error(const pic_batch *bt) { return bt ? bt->err.c_str() : "null batch"; }

int64_t pic_batch_num_particles(const pic_batch *bt, int inst) {
  if (!bt || inst < 0 || inst >= bt->B) return -1;
  return bt->np[inst];
}

int pic_batch_set_instance(pic_batch *bt, int inst, const int32_t *species, const double *x,
                           const double *u, const double *w, const double *A, const double *U) {
  if (!bt || inst < 0 || inst >= bt->B) return PIC_EARG;
  const int64_t n = bt->np[inst];
  const size_t n3 = 3 * (size_t)bt->inst[inst].nx;
  if (n > 0 && (!x || !u || !w)) return PIC_EARG;
  pic_batch::Stage &s = bt->stage[inst];
  s.sp.assign(n, 0);
  if (species)
    for (int64_t i = 0; i < n; i++) {
      if (species[i] < 0 || species[i] >= bt->nspecies) return PIC_EARG;
      s.sp[i] = species[i];
    }
  s.x.assign(x, x + n);
  s.u.assign(u, u + 3 * n);
  s.w.assign(w, w + n);
  if (A) s.A.assign(A, A + n3);
  else s.A.assign(n3, 0.0);
  if (U) s.U.assign(U, U + n3);
  else s.U.assign(n3, 0.0);
  s.set = true;
  bt->started = 0;
  return PIC_OK;
}

int pic_batch_start(pic_batch *bt, pic_report *reports) {
  if (!bt) return PIC_EARG;
  for (int b = 0; b < bt->B; b++)
    if (!bt->stage[b].set) {
      bt->err = "pic_batch_start: instance " + std::to_string(b) + " has no data";
      return PIC_ESTATE;
    }
  BCK(cudaStreamSynchronize(bt->st));
  std::map<std::tuple<int, double, double>, pic_ctx *> ctxs;
  int e = PIC_OK;
  const size_t R = bt->rsize;
  for (int b = 0; b < bt->B && !e; b++) {
    const BInst &in = bt->inst[b];
    const auto key = std::make_tuple(in.nx, in.L, in.x0);
    pic_ctx *c = ctxs[key];
    if (!c) {
      pic_grid g;
      std::memset(&g, 0, sizeof g);
      g.dim = 1;
      g.n[0] = in.nx;
      g.n[1] = 1;
      g.n[2] = 1;
      g.L[0] = in.L;
      g.L[1] = 1.0;
      g.L[2] = 1.0;
      g.x0[0] = in.x0;
      pic_options o = bt->opt;
      o.sort_every = 0;  // keep the load order
      o.cuda_stream = (void *)bt->st;
      pic_species sp[PIC_MAX_SPECIES];
      for (int s = 0; s < bt->nspecies; s++) {
        sp[s].q = bt->qs[s];
        sp[s].m = bt->ms[s];
      }
      if ((e = pic_init(&c, &g, sp, bt->nspecies, bt->dt, &o))) {
        bt->err = "pic_batch_start: pic_init failed";
        break;
      }
      ctxs[key] = c;
    }
    pic_batch::Stage &s = bt->stage[b];
    const int64_t n = bt->np[b];
    pic_report rep;
    if ((e = pic_set_particles(c, n, s.sp.data(), s.x.data(), s.u.data(), 0, s.w.data(), 0)) ||
        (e = pic_set_potentials(c, s.A.data(), s.U.data(), 0)) || (e = pic_start(c, &rep))) {
      bt->err = std::string("pic_batch_start: ") + pic_last_error(c);
      break;
    }
    bt->E0[b] = rep.E_tot;
    if (reports) reports[b] = rep;
    // copy the prepared state (load order: the context does not sort here)
    const int64_t p0 = in.pbeg;
    const int N = in.nx;
    std::vector<int64_t> ids(n);
    for (int64_t i = 0; i < n; i++) ids[i] = i;
    cudaError_t ce = cudaSuccess;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
      if (ce == cudaSuccess && bytes)
        ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, bt->st);
    };
    cp(bt->cell + p0, c->cell, sizeof(int32_t) * n);
    cp((char *)bt->off + R * p0, c->off, R * n);
    for (int q = 0; q < 3; q++)
      cp((char *)bt->P + R * (q * bt->cap + p0), (char *)c->P + R * q * c->cap, R * n);
    cp(bt->w + p0, c->w, sizeof(double) * n);
    cp(bt->sp + p0, c->sp, sizeof(int32_t) * n);
    cp(bt->id + p0, ids.data(), sizeof(int64_t) * n);
    cp(bt->phi_h + in.moff, c->phi_h, sizeof(double2) * N);
    cp(bt->psi_h + in.moff, c->psi_h, sizeof(double2) * N);
    cp(bt->rho_h + in.moff, c->rho_h, sizeof(double2) * N);
    cp(bt->A_h + 3 * in.moff, c->A_h, sizeof(double2) * 3 * N);
    cp(bt->U_h + 3 * in.moff, c->U_h, sizeof(double2) * 3 * N);
    cp(bt->A_real + 3 * in.moff, c->A_real, sizeof(double) * 3 * N);
    cp(bt->J_acc + 3 * in.moff, c->J_acc, sizeof(double) * 3 * N);
    if (bt->rsize == 4) cp((float *)bt->AT + 3 * in.moff, c->A_real_f, sizeof(float) * 3 * N);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(bt->st);  // ids and the context are reused
    if (ce != cudaSuccess) {
      bt->err = std::string("pic_batch_start: ") + cudaGetErrorString(ce);
      e = PIC_ECUDA;
    }
  }
  for (auto &kv : ctxs)
    if (kv.second) pic_free(kv.second);
  if (e) return e;
  if (bt->opt.sort_every > 0 && (e = b_sort(bt))) return e;
  BCK(cudaStreamSynchronize(bt->st));
  bt->started = 1;
  bt->steps_done = 0;
  return PIC_OK;
}

int pic_batch_step(pic_batch *bt, double tol, pic_report *reports) {
  if (!bt) return PIC_EARG;
  TraceRange trace("pic_batch_step");
  if (!bt->started) {
    bt->err = "pic_batch_step before pic_batch_start";
    return PIC_ESTATE;
  }
  double tr, ta, itr, ita;
  b_tolerances(bt, tol, &tr, &ta, &itr, &ita);
  int e = bt->rsize == 8 ? b_step_start<double>(bt) : b_step_start<float>(bt);
  if (e) return e;
  if ((e = b_rounds(bt, tr, ta, itr, ita))) return e;
  if (bt->rsize == 8) {
    if ((e = b_commit_diag<double>(bt)) || (e = b_diag<double>(bt))) return e;
  } else {
    if ((e = b_commit_diag<float>(bt)) || (e = b_diag<float>(bt))) return e;
  }
  BCK(cudaMemcpyAsync(bt->h_state, bt->d_state, sizeof(BState) * bt->B, cudaMemcpyDeviceToHost,
                      bt->st));
  BCK(cudaMemcpyAsync(bt->h_loop, bt->d_loop, sizeof(BLoop), cudaMemcpyDeviceToHost, bt->st));
  BCK(cudaStreamSynchronize(bt->st));
  if (bt->graph_ok == 1) {  // the host-driven rounds counted their own launches
    const long long rounds = bt->h_loop->rounds;
    bt->launches += rounds * (bt->nblocks > 0 ? 7 : 5);
    if (bt->nblocks > 0) bt->map_launches += 2 * rounds;
  }
  if (bt->h_loop->overflow) {
    bt->err = "pic_batch_step: the outer control did not finish within its round limit";
    return PIC_EOUTER;
  }
  int status = PIC_OK;
  for (int b = 0; b < bt->B; b++) {
    const BState &s = bt->h_state[b];
    const double *d = bt->h_diag + 4 * b;
    bt->pushes += (long long)bt->np[b] * s.map_evals;
    bt->inner_iters += (long long)s.inner_total;
    bt->pieces += (long long)s.pieces_total;
    bt->refined += (long long)s.refined_total;
    if (s.status != PIC_OK && status == PIC_OK) {
      status = s.status;
      bt->err = "instance " + std::to_string(b) + ": " + why_text(s.why);
    }
    if (reports) {
      pic_report &Rp = reports[b];
      std::memset(&Rp, 0, sizeof Rp);
      Rp.status = s.status;
      Rp.outer_iters = s.outer_iters;
      Rp.map_evals = s.map_evals;
      Rp.res_scaled_rms = s.res_srms;
      Rp.res_scaled_max = s.res_smax;
      Rp.K = d[0];
      Rp.W = d[1];
      Rp.E_tot = d[0] + d[1];
      Rp.gauss_rms = d[2];
      Rp.lorenz_rms = d[3];
      Rp.rel_dE = bt->E0[b] != 0.0 ? (Rp.E_tot - bt->E0[b]) / bt->E0[b] : 0.0;
      if (s.status == PIC_OK) {
        Rp.work_residual = bt->dt * (s.work_p - s.work_mesh);
        Rp.chain_rms = bt->np[b] ? std::sqrt(s.chain / (3.0 * bt->np[b])) : 0.0;
        Rp.inner_max = s.inner_max;
        Rp.inner_mean = bt->np[b] ? (double)s.inner_sum / bt->np[b] : 0.0;
        Rp.refined = (int)s.refined_final;
      }
    }
  }
  bt->steps_done++;
  if (bt->opt.sort_every > 0 && bt->steps_done % bt->opt.sort_every == 0) {
    if ((e = b_sort(bt))) return e;
    BCK(cudaStreamSynchronize(bt->st));
  }
  return status;
}

int pic_batch_get_particles(pic_batch *bt, int inst, double *x, double *P, double *w,
                            int32_t *species) {
  if (!bt || inst < 0 || inst >= bt->B) return PIC_EARG;
  const BInst &in = bt->inst[inst];
  const int64_t n = bt->np[inst];
  if (n == 0) return PIC_OK;
  double *dx = bt->d_out, *dP = dx + n, *dw = dP + 3 * n;
  int32_t *dsp = (int32_t *)(dw + n);
  const int nb = (int)((n + kPT - 1) / kPT);
  if (bt->rsize == 8)
    k_bexport<double><<<nb, kPT, 0, bt->st>>>(bt->cap, bt->cell, (const double *)bt->off,
                                              (const double *)bt->P, bt->w, bt->sp, bt->id, in,
                                              dx, dP, dw, dsp);
  else
    k_bexport<float><<<nb, kPT, 0, bt->st>>>(bt->cap, bt->cell, (const float *)bt->off,
                                             (const float *)bt->P, bt->w, bt->sp, bt->id, in, dx,
                                             dP, dw, dsp);
  BKCHECK();
  if (x) BCK(cudaMemcpyAsync(x, dx, sizeof(double) * n, cudaMemcpyDeviceToHost, bt->st));
  if (P) BCK(cudaMemcpyAsync(P, dP, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, bt->st));
  if (w) BCK(cudaMemcpyAsync(w, dw, sizeof(double) * n, cudaMemcpyDeviceToHost, bt->st));
  if (species)
    BCK(cudaMemcpyAsync(species, dsp, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, bt->st));
  BCK(cudaStreamSynchronize(bt->st));
  return PIC_OK;
}

int pic_batch_get_potentials(pic_batch *bt, int inst, double *phi, double *psi, double *A,
                             double *U, double *rho, double *J) {
  if (!bt || inst < 0 || inst >= bt->B) return PIC_EARG;
  const BInst &in = bt->inst[inst];
  const int N = in.nx;
  k_bto_real<<<1, kBT, field_smem(bt), bt->st>>>(in, bt->phi_h, bt->psi_h, bt->rho_h, bt->A_h,
                                                  bt->U_h, bt->tw, bt->d_out);
  BKCHECK();
  const double *o = bt->d_out;
  auto get = [&](double *dst, const double *src, size_t cnt) -> cudaError_t {
    return dst ? cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToHost, bt->st)
               : cudaSuccess;
  };
  BCK(get(phi, o, N));
  BCK(get(psi, o + N, N));
  BCK(get(rho, o + 2 * N, N));
  BCK(get(A, o + 3 * N, 3 * (size_t)N));
  BCK(get(U, o + 6 * N, 3 * (size_t)N));
  BCK(get(J, bt->J_acc + 3 * in.moff, 3 * (size_t)N));
  BCK(cudaStreamSynchronize(bt->st));
  return PIC_OK;
}

int pic_batch_get_stats(const pic_batch *bt, pic_stats *out) {
  if (!bt || !out) return PIC_EARG;
  std::memset(out, 0, sizeof *out);
  out->launches = bt->launches;
  out->map_launches = bt->map_launches;
  out->map_ms = 0.0;
  out->pushes = bt->pushes;
  out->inner_iters = bt->inner_iters;
  out->pieces = bt->pieces;
  out->refined = bt->refined;
  return PIC_OK;
}

int pic_batch_reset_stats(pic_batch *bt) {
  if (!bt) return PIC_EARG;
  bt->launches = bt->map_launches = bt->pushes = bt->inner_iters = bt->pieces = bt->refined = 0;
  return PIC_OK;
}

}  // extern "C"
