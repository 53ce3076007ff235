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
  // exact snapshot of the accepted state (the device arrays themselves, in
  // device memory)
  struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
      if (p) cudaFree(p);
    }
  } snap;
  int e;
  CK(cudaMalloc(&snap.p, state_snapshot_bytes(ctx)));
  if ((e = state_snapshot(ctx, snap.p))) return e;
  const int sort0 = ctx->opt.sort_every;
  const long long steps0 = ctx->steps_done;
  const double E0 = ctx->E0;
  const int64_t np0 = ctx->np;
  // every candidate starts from the snapshot, sorted by cell when it sorts
  // at all (as pic_start leaves the particles)
  auto restore = [&](int sort_every, bool sort_now) -> int {
    int r = state_restore(ctx, snap.p, np0, steps0, sort_every, E0);
    if (r) return r;
    return sort_now && sort_every > 0 ? particles_sort(ctx) : PIC_OK;
  };
  cudaEvent_t ea, eb;
  CK(cudaEventCreate(&ea));
  CK(cudaEventCreate(&eb));
  int best = -1, status = PIC_OK;
  double best_ms = INFINITY;
  for (int k = 0; k < ncand && status == PIC_OK; k++) {
    if ((status = restore(cand[k], true))) break;
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
  // the state exactly as it was (same bits, same particle order, same step
  // count), with the chosen interval; the statistics without the tuning steps
  const int r = restore(status == PIC_OK ? best : sort0, false);
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
