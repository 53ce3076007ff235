// fft.cu -- batched radix-2 complex FFT along the axes of the periodic mesh.
//
// The CN potential update of Sec. 2.3 is solved mode by mode in Fourier
// space (Sec. 4.5), so every map evaluation transforms a handful of mesh
// arrays forward and back.  Meshes here are small (64 .. 512^2 nodes), so
// one CTA transforms several whole lines in shared memory: it loads them
// bit-reversed (coalesced across adjacent lines for strided axes), runs
// log2(n) decimation-in-time butterfly stages, and stores them back in
// natural order.  Transforms are unnormalised in both directions; callers
// apply 1/Ng.
#include "pic_internal.cuh"

#include <cmath>
#include <vector>

namespace {

constexpr int kFftThreads = 256;
constexpr int kFftSmemElems = 4096;  // double2 per CTA (64 KB)

__global__ void __launch_bounds__(kFftThreads)
k_fft_axis(double2 *__restrict__ data, int Ng, int N, int logN, int stride, int lines,
           int lpb, const double2 *__restrict__ tw, int inverse) {
  extern __shared__ double2 sm[];
  double2 *base_data = data + (size_t)blockIdx.y * Ng;
  const int line0 = blockIdx.x * lpb;
  const int nl = min(lpb, lines - line0);
  const int tot = nl * N;
  // load, bit-reversed within each line
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    int b, k;
    if (stride == 1) { b = t / N; k = t - b * N; }
    else { k = t / nl; b = t - k * nl; }
    int ln = line0 + b;
    int inner = ln % stride, outer = ln / stride;
    size_t addr = (size_t)inner + (size_t)outer * stride * N + (size_t)k * stride;
    int kr = (int)(__brev((unsigned)k) >> (32 - logN));
    sm[b * N + kr] = base_data[addr];
  }
  __syncthreads();
  const int half = N >> 1;
  for (int h = 1; h < N; h <<= 1) {
    const int tstep = N / (2 * h);
    for (int t = threadIdx.x; t < nl * half; t += blockDim.x) {
      int b = t / half, j = t - b * half;
      int grp = j / h, pos = j - grp * h;
      int i0 = b * N + grp * 2 * h + pos, i1 = i0 + h;
      double2 wv = tw[pos * tstep];
      if (inverse) wv.y = -wv.y;
      double2 x0 = sm[i0], x1 = sm[i1];
      double2 y;
      y.x = wv.x * x1.x - wv.y * x1.y;
      y.y = wv.x * x1.y + wv.y * x1.x;
      sm[i0] = make_double2(x0.x + y.x, x0.y + y.y);
      sm[i1] = make_double2(x0.x - y.x, x0.y - y.y);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    int b, k;
    if (stride == 1) { b = t / N; k = t - b * N; }
    else { k = t / nl; b = t - k * nl; }
    int ln = line0 + b;
    int inner = ln % stride, outer = ln / stride;
    size_t addr = (size_t)inner + (size_t)outer * stride * N + (size_t)k * stride;
    base_data[addr] = sm[b * N + k];
  }
}

}  // namespace

int fft_init(pic_ctx *ctx) {
  for (int a = 0; a < 3; a++) ctx->tw[a] = nullptr;
  for (int a = 0; a < ctx->g.dim; a++) {
    int N = ctx->g.n[a];
    std::vector<double2> h(N);
    for (int k = 0; k < N; k++) {
      // exp(-2 pi i k / N); exact quarter points avoid roundoff in the table
      double c, s;
      if (4 * k % N == 0) {
        int q = 4 * k / N;
        c = (q == 0) ? 1.0 : (q == 2 ? -1.0 : 0.0);
        s = (q == 1) ? 1.0 : (q == 3 ? -1.0 : 0.0);
      } else {
        double th = 2.0 * M_PI * (double)k / (double)N;
        c = std::cos(th);
        s = std::sin(th);
      }
      h[k] = make_double2(c, -s);
    }
    CK(cudaMalloc(&ctx->tw[a], sizeof(double2) * N));
    CK(cudaMemcpy(ctx->tw[a], h.data(), sizeof(double2) * N, cudaMemcpyHostToDevice));
  }
  CK(cudaFuncSetAttribute(k_fft_axis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          kFftSmemElems * (int)sizeof(double2)));
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev));
  if (ctx->num_sms < 1) ctx->num_sms = 1;
  return PIC_OK;
}

int fft_nd(pic_ctx *ctx, double2 *data, int batch, int sign) {
  const Geom &g = ctx->g;
  int stride = 1;
  for (int a = 0; a < g.dim; a++) {
    int N = g.n[a];
    int lines = g.Ng / N;
    // lines per CTA: enough CTAs for two waves over the SMs, whole lines in
    // shared memory, and (for strided axes) lines adjacent in memory
    int lpb = (int)(((long long)lines * batch) / (2LL * ctx->num_sms));
    if (lpb > kFftSmemElems / N) lpb = kFftSmemElems / N;
    if (lpb > lines) lpb = lines;
    if (a > 0 && lpb > stride) lpb = stride;
    if (lpb < 1) lpb = 1;
    int p2 = 1;
    while (p2 * 2 <= lpb) p2 *= 2;
    lpb = p2;
    int threads = lpb * N / 2;
    threads = threads < 32 ? 32 : (threads > kFftThreads ? kFftThreads : (threads + 31) / 32 * 32);
    dim3 grid((lines + lpb - 1) / lpb, batch);
    size_t smem = sizeof(double2) * (size_t)lpb * N;
    k_fft_axis<<<grid, threads, smem, ctx->st>>>(data, g.Ng, N, g.logn[a], stride, lines, lpb,
                                                 ctx->tw[a], sign > 0 ? 1 : 0);
    KCHECK();
    stride *= N;
  }
  return PIC_OK;
}
