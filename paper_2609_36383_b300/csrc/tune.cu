// tune.cu -- pic_tune_sort(): the autotuner of the counting-sort interval.
//
// The particle map reads its gather records by cell, so particles sorted by
// cell read neighbouring records in neighbouring threads, and a warp's
// orbits share stencil nodes.  Particles drift out of that order every step;
// re-sorting costs a histogram, a scan and a permutation of every particle
// array.  The best interval depends on the drift per step and on the map's
// cost, so it is measured: each candidate runs the same steps from the same
// checkpoint, timed with CUDA events on the context's stream, and the
// fastest is kept.  (The particle kernels' CTA size is not tuned: the
// piece-count grouping and the deposit window are built for 128 threads.)
#include "pic_internal.cuh"

#include <cmath>
#include <vector>

extern "C" int pic_tune_sort(pic_ctx *ctx, double tol, int steps, const int *cand, int ncand,
                             int *best_out, double *ms_out) {
  if (!ctx || !cand || ncand < 1 || ncand > 64 || steps < 1 || steps > 1000) return PIC_EARG;
  for (int k = 0; k < ncand; k++)
    if (cand[k] < 0) {
      ctx->err = "pic_tune_sort: negative sort interval";
      return PIC_EARG;
    }
  if (!ctx->started) {
    ctx->err = "pic_tune_sort before pic_start";
    return PIC_ESTATE;
  }
  // the statistics before anything here launches (restored at the end)
  const long long st_l = ctx->launches, st_ml = ctx->map_launches, st_p = ctx->pushes,
                  st_i = ctx->inner_iters, st_pc = ctx->pieces, st_r = ctx->refined;
  const double st_ms = ctx->map_ms;
  const int64_t n = ctx->np;
  const int d = ctx->g.dim;
  const size_t Ng = ctx->g.Ng;
  // checkpoint of the accepted state (host copies, load order)
  std::vector<double> x((size_t)d * n), P(3 * (size_t)n), w(n), phi(Ng), psi(Ng), A(3 * Ng),
      U(3 * Ng), rho(Ng), J(3 * Ng);
  std::vector<int32_t> sp(n);
  int e;
  if ((e = pic_get_particles(ctx, x.data(), P.data(), w.data(), sp.data(), 0))) return e;
  if ((e = pic_get_potentials(ctx, phi.data(), psi.data(), A.data(), U.data(), rho.data(),
                              J.data(), 0)))
    return e;
  const double E0 = ctx->E0;
  const long long steps_done = ctx->steps_done;
  const int sort0 = ctx->opt.sort_every;
  // restore the checkpoint; particles come back in load order and are
  // sorted once when an interval is set, as pic_start sorts them
  auto restore = [&](int sort_every) -> int {
    int r = pic_set_state(ctx, n, sp.data(), x.data(), P.data(), w.data(), phi.data(),
                          psi.data(), A.data(), U.data(), rho.data(), J.data(), E0, 0);
    if (r) return r;
    ctx->opt.sort_every = sort_every;
    return sort_every > 0 ? particles_sort(ctx) : PIC_OK;
  };
  cudaEvent_t ea, eb;
  CK(cudaEventCreate(&ea));
  CK(cudaEventCreate(&eb));
  int best = -1, status = PIC_OK;
  double best_ms = INFINITY;
  for (int k = 0; k < ncand && status == PIC_OK; k++) {
    if ((status = restore(cand[k]))) break;
    ctx->steps_done = 0;  // every candidate starts in the same phase
    if (cudaEventRecord(ea, ctx->st) != cudaSuccess) {
      status = PIC_ECUDA;
      break;
    }
    for (int s = 0; s < steps && status == PIC_OK; s++) {
      pic_report R;
      status = pic_step(ctx, tol, &R);
    }
    if (status != PIC_OK) break;
    float ms = 0.0f;
    if (cudaEventRecord(eb, ctx->st) != cudaSuccess || cudaEventSynchronize(eb) != cudaSuccess ||
        cudaEventElapsedTime(&ms, ea, eb) != cudaSuccess) {
      status = PIC_ECUDA;
      break;
    }
    const double per = ms / steps;
    if (ms_out) ms_out[k] = per;
    if (per < best_ms) {
      best_ms = per;
      best = cand[k];
    }
  }
  cudaEventDestroy(ea);
  cudaEventDestroy(eb);
  // the state as it was, with the chosen interval; the statistics without
  // the tuning steps
  const int r = restore(status == PIC_OK ? best : sort0);
  ctx->steps_done = steps_done;
  ctx->launches = st_l;
  ctx->map_launches = st_ml;
  ctx->pushes = st_p;
  ctx->inner_iters = st_i;
  ctx->pieces = st_pc;
  ctx->refined = st_r;
  ctx->map_ms = st_ms;
  if (status != PIC_OK) return status;
  if (r) return r;
  if (best_out) *best_out = best;
  return PIC_OK;
}
