// peak.cu -- FMA-throughput microbenchmark behind pic_fma_throughput().
//
// The particle map is bound by FP64 (or, in the mixed path, FP32) arithmetic,
// and no measured figure exists for either pipe, so the library
// measures them: every thread runs kChains independent FMA chains for `iters`
// iterations (enough independent work to hide the pipe latency), the grid
// has 8 CTAs of 256 threads per SM, and the result is stored so the compiler
// keeps the loop.
#include "pic_internal.cuh"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma(T *out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run(double *flops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PIC_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PIC_ECUDA;
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 4096 : 65536;
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return PIC_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma<T><<<blocks, threads>>>(out, 16, (T)0.999, (T)1e-6);  // warm-up
  cudaEventRecord(e0);
  k_fma<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)1e-6);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.0f) return PIC_ECUDA;
  *flops = 2.0 * kChains * (double)iters * blocks * threads / (ms * 1e-3);
  return PIC_OK;
}

}  // namespace

extern "C" int pic_fma_throughput(int precision, double *flops_per_s) {
  if (!flops_per_s) return PIC_EARG;
  return precision == PIC_MIXED ? run<float>(flops_per_s) : run<double>(flops_per_s);
}
