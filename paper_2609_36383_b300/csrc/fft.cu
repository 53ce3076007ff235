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

// Every size here is a power of two (line length N = 2^logN, the stride of
// the axis 2^logS, lines per CTA), so the index arithmetic uses shifts and
// masks rather than integer divisions.
__global__ void __launch_bounds__(kFftThreads)
k_fft_axis(double2 *__restrict__ data, int Ng, int N, int logN, int logS, int lines, int lpb,
           int loglpb, const double2 *__restrict__ tw, int inverse) {
  extern __shared__ double2 sm[];
  double2 *base_data = data + (size_t)blockIdx.y * Ng;
  const int line0 = blockIdx.x * lpb;
  const int nl = min(lpb, lines - line0);
  const int tot = nl * N;
  const int smask = (1 << logS) - 1, nmask = N - 1;
  // load, bit-reversed within each line
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    int b, k;
    if (logS == 0) { b = t >> logN; k = t & nmask; }
    else { k = t >> loglpb; b = t & (lpb - 1); }
    const int ln = line0 + b;
    const int inner = ln & smask, outer = ln >> logS;
    const size_t addr = (size_t)inner + ((size_t)outer << (logS + logN)) + ((size_t)k << logS);
    const int kr = (int)(__brev((unsigned)k) >> (32 - logN));
    sm[(b << logN) + kr] = base_data[addr];
  }
  __syncthreads();
  const int logHalf = logN - 1;
  for (int lh = 0; lh < logN; lh++) {
    const int h = 1 << lh;
    const int tshift = logN - 1 - lh;  // twiddle stride N / (2h)
    for (int t = threadIdx.x; t < (nl << logHalf); t += blockDim.x) {
      const int b = t >> logHalf, j = t & ((1 << logHalf) - 1);
      const int grp = j >> lh, pos = j & (h - 1);
      const int i0 = (b << logN) + (grp << (lh + 1)) + pos, i1 = i0 + h;
      double2 wv = tw[pos << tshift];
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
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    int b, k;
    if (logS == 0) { b = t >> logN; k = t & nmask; }
    else { k = t >> loglpb; b = t & (lpb - 1); }
    const int ln = line0 + b;
    const int inner = ln & smask, outer = ln >> logS;
    const size_t addr = (size_t)inner + ((size_t)outer << (logS + logN)) + ((size_t)k << logS);
    base_data[addr] = sm[(b << logN) + k];
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
    int logS = 0, loglpb = 0;
    while ((1 << logS) < stride) logS++;
    while ((1 << loglpb) < lpb) loglpb++;
    k_fft_axis<<<grid, threads, smem, ctx->st>>>(data, g.Ng, N, g.logn[a], logS, lines, lpb,
                                                 loglpb, ctx->tw[a], sign > 0 ? 1 : 0);
    KCHECK();
    stride *= N;
  }
  return PIC_OK;
}
