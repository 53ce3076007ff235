// noalloc.cu -- pic_kinetic_energy_noalloc(): the kinetic-energy reduction of
// a particle set, for callers that cannot allocate GPU memory.
//
// Some callers may not call cudaMalloc at all.  A memory arena or pool may
// own the whole device, an allocation may synchronize the device inside a
// latency-critical loop, or a framework's policy may forbid allocations on
// its hot path.  This entry point keeps its scratch (the per-block partial
// sums and the final result) in a fixed file-scope device array instead, so
// it allocates nothing.  The caller still passes the inputs (device arrays)
// and receives the result in host memory.
//
// The computation is the same sum the context reports as K: for every
// particle, p = P - q A_h(x) and K_i = m kappa^2 (gamma - 1), evaluated as
// |p|^2 / (m (gamma + 1)).  Positions arrive as absolute coordinates, so the
// kernel forms the nearest node and offset itself.
#include "pic_internal.cuh"

#include <atomic>
#include <cmath>

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = 16384;  // at most kNaMaxBlocks * kNaThreads particles
static_assert((long long)kNaMaxBlocks * kNaThreads == PIC_NOALLOC_MAX_PARTICLES,
              "PIC_NOALLOC_MAX_PARTICLES must match the scratch size");
constexpr int kNaMaxDevices = 64;

// Block partials, one slot for the finished sum, and one error word (set to
// 1 by a thread that met a species index out of range): 16386 doubles.
constexpr int kNaSum = kNaMaxBlocks, kNaErr = kNaMaxBlocks + 1;
static __device__ __align__(256) double g_noalloc_scratch[kNaMaxBlocks + 2];

// Device address of g_noalloc_scratch, looked up once per device.  Two
// threads that make their first call at the same time both look it up and
// store the same value.
std::atomic<double *> g_scratch_ptr[kNaMaxDevices];

struct NaGeom {
  int dim, n[3], mask[3], n0, n01, Ng, nspecies;
  double x0[3], inv_dx[3];
  double qs[PIC_MAX_SPECIES], ms[PIC_MAX_SPECIES];
  double kappa;
};

__device__ __forceinline__ void na_weights(double t, double S[3]) {
  double a = 0.5 - t, b = 0.5 + t;
  S[0] = 0.5 * a * a;
  S[1] = 0.75 - t * t;
  S[2] = 0.5 * b * b;
}

__global__ void __launch_bounds__(kNaThreads)
k_kinetic_noalloc(int64_t n, const int32_t *__restrict__ sp, const double *__restrict__ x,
                  const double *__restrict__ P, const double *__restrict__ w,
                  const double *__restrict__ A, NaGeom g, double *__restrict__ parts) {
  const int64_t i = blockIdx.x * (int64_t)kNaThreads + threadIdx.x;
  double k = 0.0;
  if (i < n) {
    int cell[3] = {0, 0, 0};
    double S[3][3];
    for (int l = 0; l < 3; l++) S[l][0] = S[l][2] = 0.0, S[l][1] = 1.0;
    for (int l = 0; l < g.dim; l++) {
      double u = (x[l * n + i] - g.x0[l]) * g.inv_dx[l];
      double nn = (double)g.n[l];
      u -= nn * floor(u / nn);
      double c = floor(u + 0.5);
      cell[l] = (int)c & g.mask[l];
      na_weights(u - c, S[l]);
    }
    double Ax[3] = {0.0, 0.0, 0.0};
    for (int oz = 0; oz < (g.dim > 2 ? 3 : 1); oz++)
      for (int oy = 0; oy < (g.dim > 1 ? 3 : 1); oy++)
        for (int ox = 0; ox < 3; ox++) {
          int gi = (cell[0] + ox - 1) & g.mask[0];
          if (g.dim > 1) gi += g.n0 * ((cell[1] + oy - 1) & g.mask[1]);
          if (g.dim > 2) gi += g.n01 * ((cell[2] + oz - 1) & g.mask[2]);
          double s = S[0][ox] * (g.dim > 1 ? S[1][oy] : 1.0) * (g.dim > 2 ? S[2][oz] : 1.0);
          for (int c = 0; c < 3; c++) Ax[c] += s * A[(size_t)c * g.Ng + gi];
        }
    int s = sp ? sp[i] : 0;
    if (s < 0 || s >= g.nspecies) {  // never index the tables with it
      parts[kNaErr] = 1.0;
      s = 0;
    }
    double q = w[i] * g.qs[s], m = w[i] * g.ms[s];
    double p2 = 0.0;
    for (int c = 0; c < 3; c++) {
      double p = P[c * n + i] - q * Ax[c];
      p2 += p * p;
    }
    double gam = sqrt(1.0 + p2 / (m * m * g.kappa * g.kappa));
    k = p2 / (m * (gam + 1.0));
  }
  __shared__ double sh[kNaThreads / 32];
  for (int o = 16; o > 0; o >>= 1) k += __shfl_down_sync(0xffffffffu, k, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = k;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int v = 0; v < kNaThreads / 32; v++) t += sh[v];
    parts[blockIdx.x] = t;  // every used slot is overwritten: no clearing needed
  }
}

// Sums the nb partials in a fixed order into parts[kNaSum].
__global__ void k_kinetic_noalloc_final(double *parts, int nb) {
  __shared__ double sh[kNaThreads];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += kNaThreads) s += parts[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = kNaThreads / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) parts[kNaSum] = sh[0];
}

bool na_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" int pic_kinetic_energy_noalloc(const pic_grid *grid, const pic_species *species,
                                          int nspecies, double kappa, int64_t n,
                                          const int32_t *sp, const double *x, const double *P,
                                          const double *w, const double *A, double *K_out,
                                          void *cuda_stream) {
  if (!grid || !species || !K_out || nspecies < 1 || nspecies > PIC_MAX_SPECIES ||
      !(kappa > 0.0) || n < 0 || grid->dim < 1 || grid->dim > 3)
    return PIC_EARG;
  if (n > (int64_t)kNaMaxBlocks * kNaThreads) return PIC_ETOOBIG;  // beyond the fixed scratch
  if (n > 0 && (!x || !P || !w || !A)) return PIC_EARG;
  NaGeom g;
  g.dim = grid->dim;
  g.Ng = 1;
  for (int l = 0; l < 3; l++) {
    bool act = l < grid->dim;
    if (act && (!na_pow2(grid->n[l]) || grid->n[l] < 4 || grid->n[l] > 4096 ||
                !(grid->L[l] > 0.0)))
      return PIC_EARG;
    g.n[l] = act ? grid->n[l] : 1;
    g.mask[l] = g.n[l] - 1;
    g.x0[l] = act ? grid->x0[l] : 0.0;
    g.inv_dx[l] = act ? grid->n[l] / grid->L[l] : 1.0;
    g.Ng *= g.n[l];
  }
  g.n0 = g.n[0];
  g.n01 = g.n[0] * g.n[1];
  for (int s = 0; s < PIC_MAX_SPECIES; s++) {
    g.qs[s] = s < nspecies ? species[s].q : 0.0;
    g.ms[s] = s < nspecies ? species[s].m : 1.0;
    if (s < nspecies && !(species[s].m > 0.0)) return PIC_EARG;
  }
  g.kappa = kappa;
  g.nspecies = nspecies;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return PIC_ECUDA;
  // set-up, once per device, with that device current: the array's name is
  // only a host-side stand-in, so fetch the device address it refers to
  double *parts = g_scratch_ptr[dev].load();
  if (!parts) {
    if (cudaGetSymbolAddress((void **)&parts, g_noalloc_scratch) != cudaSuccess || !parts)
      return PIC_ECUDA;
    g_scratch_ptr[dev].store(parts);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the error word keeps the previous call's value: clear it
  if (cudaMemsetAsync(parts + kNaErr, 0, sizeof(double), st) != cudaSuccess) return PIC_ECUDA;
  int nb = (int)((n + kNaThreads - 1) / kNaThreads);
  if (nb > 0) {
    k_kinetic_noalloc<<<nb, kNaThreads, 0, st>>>(n, sp, x, P, w, A, g, parts);
    if (cudaGetLastError() != cudaSuccess) return PIC_ECUDA;
  }
  k_kinetic_noalloc_final<<<1, kNaThreads, 0, st>>>(parts, nb);
  if (cudaGetLastError() != cudaSuccess) return PIC_ECUDA;
  double res[2];  // the sum and the error word, adjacent in the scratch
  if (cudaMemcpyAsync(res, parts + kNaSum, sizeof res, cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return PIC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PIC_ECUDA;
  if (res[1] != 0.0) return PIC_EARG;
  *K_out = res[0];
  return PIC_OK;
}
