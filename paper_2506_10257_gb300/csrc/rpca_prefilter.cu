// rpca_prefilter.cu -- the frame pre-filter of the in vivo reference (Sec. III,
// "Applying the RPCA method"): frames that correlate below a limit with every
// neighbouring frame are excluded, and a temporal moving average over a window
// of frames runs over the kept frames before the RPCA solve.
//
// Readings (the paper gives no formula): the correlation of frames t and t+1
// is Pearson's coefficient over all pixels; frame t is kept when it reaches
// the limit with at least one neighbour (a single frame is kept); the moving
// average covers whole windows of kept frames only (output j = mean of kept
// frames j .. j+w-1); a frame without variance correlates 0.
//
// Three launches, all stream-ordered, no host round trip:
//   pf_stats_kernel   grid (chunks, T): per frame t and pixel chunk, FP64 sums
//                     of y_t, y_t^2 and y_t y_{t+1} with y_t = x_t - x_t[0]
//                     (the shift keeps the centred moments free of
//                     cancellation; FP32 inputs make y and the products exact
//                     in FP64);
//   pf_decide_kernel  one CTA: sums the chunks in fixed order, forms the
//                     neighbour correlations, keeps frames, writes the counts;
//   pf_average_kernel a thread per (pixel, 16 output frames): the window sum
//                     in FP64, formed directly for the first output and slid
//                     for the rest (exact for FP32 inputs of similar
//                     magnitude), each output frame written as FP32.
//
// The temporal high-pass that Sec. IV suggests before RPCA (no filter is
// defined there) is read as the complement of the same moving average: output
// j = kept frame j + (w-1)/2 (rounded down) minus the mean of window j, formed
// in FP64 from the same sliding sum and rounded once to FP32.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/rpca.h"

namespace {

constexpr int kPfThreads = 256;
constexpr int kPfChunkPix = 8 * kPfThreads;  // pixels of a stats CTA
constexpr int kPfMaxChunks = 256;

int pf_chunks(int64_t m) {
  const int64_t c = (m + kPfChunkPix - 1) / kPfChunkPix;
  return (int)(c < kPfMaxChunks ? c : kPfMaxChunks);
}

__device__ __forceinline__ double pf_block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kPfThreads / 32; ++i) s += sh[i];  // fixed order
  return s;  // valid in thread 0
}

// partial[(t * nch + c) * 3 + {0, 1, 2}] = sum y_t, sum y_t^2, sum y_t y_{t+1}
__global__ void __launch_bounds__(kPfThreads) pf_stats_kernel(const float* __restrict__ X, int64_t m, int T,
                                                              double* __restrict__ partial) {
  __shared__ double sh[kPfThreads / 32];
  const int t = blockIdx.y, c = blockIdx.x, nch = gridDim.x;
  const int64_t per = (m + nch - 1) / nch;
  const int64_t p0 = (int64_t)c * per, p1 = (p0 + per < m) ? p0 + per : m;
  const float* xt = X + (int64_t)t * m;
  const bool has_next = (t + 1 < T);
  const float* xn = X + (int64_t)(has_next ? t + 1 : t) * m;
  const double at = (double)xt[0], an = (double)xn[0];
  double s1 = 0.0, s2 = 0.0, pr = 0.0;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kPfThreads) {
    const double y = (double)xt[p] - at;
    s1 += y;
    s2 = fma(y, y, s2);
    if (has_next) pr = fma(y, (double)xn[p] - an, pr);
  }
  const double r1 = pf_block_sum(s1, sh);
  const double r2 = pf_block_sum(s2, sh);
  const double r3 = pf_block_sum(pr, sh);
  if (threadIdx.x == 0) {
    double* o = partial + ((int64_t)t * nch + c) * 3;
    o[0] = r1;
    o[1] = r2;
    o[2] = r3;
  }
}

// stats in dynamic shared memory: [T][3] doubles, then T ints (keep flags)
__global__ void __launch_bounds__(kPfThreads) pf_decide_kernel(const double* __restrict__ partial, int64_t m,
                                                               int T, int nch, double corr_min, int window,
                                                               double* corr_out, int* kept, int* count) {
  extern __shared__ double pf_sh[];
  double* st = pf_sh;                                 // [T][3]
  int* keep = reinterpret_cast<int*>(pf_sh + 3 * T);  // [T]
  double* cc = pf_sh + 3 * T + (T + 1) / 2;           // [T - 1] correlations
  const double dm = (double)m;
  for (int i = threadIdx.x; i < 3 * T; i += blockDim.x) {
    const int t = i / 3, k = i % 3;
    const double* src = partial + (int64_t)t * nch * 3 + k;
    double s = 0.0;
    for (int c0 = 0; c0 < nch; c0 += 16) {
      double v[16];  // sixteen loads in flight, then added in chunk order
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = (c0 + u < nch) ? src[(int64_t)(c0 + u) * 3] : 0.0;
#pragma unroll
      for (int u = 0; u < 16; ++u) s += v[u];
    }
    st[i] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < T - 1; t += blockDim.x) {
    const double sxx = st[3 * t + 1] - st[3 * t] * st[3 * t] / dm;
    const double syy = st[3 * (t + 1) + 1] - st[3 * (t + 1)] * st[3 * (t + 1)] / dm;
    const double sxy = st[3 * t + 2] - st[3 * t] * st[3 * (t + 1)] / dm;
    const double r = (sxx > 0.0 && syy > 0.0) ? sxy / sqrt(sxx * syy) : 0.0;
    cc[t] = r;
    if (corr_out) corr_out[t] = r;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    int k = (T == 1);
    if (t > 0 && cc[t - 1] >= corr_min) k = 1;
    if (t < T - 1 && cc[t] >= corr_min) k = 1;
    keep[t] = k;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int K = 0;
    for (int t = 0; t < T; ++t)
      if (keep[t]) kept[K++] = t;
    count[0] = K;
    count[1] = (K >= window) ? K - window + 1 : 0;
  }
}

constexpr int kPfSeg = 16;  // output frames of one moving-average thread

// kept list in dynamic shared memory (T ints).  Work item (segment g, pixel p):
// output frames g*kPfSeg .. +kPfSeg-1 of pixel p; items run pixel-fastest, so
// a warp reads and writes 32 consecutive pixels of one frame.  HP: write the
// centre frame minus the mean instead of the mean.
template <bool HP>
__global__ void __launch_bounds__(kPfThreads) pf_average_kernel(const float* __restrict__ X, int64_t m, int T,
                                                                const int* __restrict__ kept,
                                                                const int* __restrict__ count, int window,
                                                                float* __restrict__ Y) {
  extern __shared__ int pf_kept[];
  for (int i = threadIdx.x; i < T; i += blockDim.x) pf_kept[i] = kept[i];
  __syncthreads();
  const int n = count[1];
  if (n <= 0) return;
  const double inv_w = 1.0 / (double)window;
  const int h = (window - 1) / 2;
  const int64_t nseg = (n + kPfSeg - 1) / kPfSeg;
  auto out = [&](int j, int64_t p, double s) {
    const double mean = s * inv_w;
    Y[(int64_t)j * m + p] = HP ? (float)((double)X[(int64_t)pf_kept[j + h] * m + p] - mean) : (float)mean;
  };
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < nseg * m;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = it % m;
    const int j0 = (int)(it / m) * kPfSeg;
    const int j1 = (j0 + kPfSeg < n) ? j0 + kPfSeg : n;
    double s = 0.0;
#pragma unroll 4
    for (int i = 0; i < window; ++i) s += (double)X[(int64_t)pf_kept[j0 + i] * m + p];
    out(j0, p, s);
    for (int j = j0 + 1; j < j1; ++j) {
      s += (double)X[(int64_t)pf_kept[j + window - 1] * m + p];
      s -= (double)X[(int64_t)pf_kept[j - 1] * m + p];
      out(j, p, s);
    }
  }
}

rpca_status prefilter_impl(const float* X, int64_t m, int32_t T, double corr_min, int32_t window, float* Y,
                           int32_t* kept, int32_t* count, double* corr, void* scratch, void* stream,
                           bool high_pass) {
  if (!X || !Y || !kept || !count || !scratch || m < 1 || T < 1 || window < 1 || !(corr_min == corr_min))
    return RPCA_ERR_ARG;
  if (((uintptr_t)X | (uintptr_t)Y) & 3u) return RPCA_ERR_ARG;
  if (T > 65535) return RPCA_ERR_UNSUPPORTED;  // one grid row per frame
  cudaStream_t s = (cudaStream_t)stream;
  const int nch = pf_chunks(m);
  double* partial = (double*)scratch;
  pf_stats_kernel<<<dim3((unsigned)nch, (unsigned)T), kPfThreads, 0, s>>>(X, m, T, partial);
  const size_t dsm = sizeof(double) * (3 * (size_t)T + (size_t)(T + 1) / 2 + (size_t)T);
  if (dsm > 48 * 1024) {
    if (cudaFuncSetAttribute(pf_decide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm) !=
        cudaSuccess)
      return RPCA_ERR_CUDA;
  }
  pf_decide_kernel<<<1, kPfThreads, dsm, s>>>(partial, m, T, nch, corr_min, window, corr, kept, count);
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                               cudaSuccess)
    return RPCA_ERR_CUDA;
  const int64_t items = m * (int64_t)((T + kPfSeg - 1) / kPfSeg);  // at most this many (segment, pixel) items
  const int64_t want = (items + kPfThreads - 1) / kPfThreads;
  const int grid = (int)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
  if (high_pass)
    pf_average_kernel<true><<<grid, kPfThreads, sizeof(int) * (size_t)T, s>>>(X, m, T, kept, count, window, Y);
  else
    pf_average_kernel<false><<<grid, kPfThreads, sizeof(int) * (size_t)T, s>>>(X, m, T, kept, count, window, Y);
  return cudaGetLastError() == cudaSuccess ? RPCA_OK : RPCA_ERR_CUDA;
}

}  // namespace

extern "C" {

size_t rpca_prefilter_scratch_bytes(int64_t m, int32_t T) {
  if (m < 1 || T < 1) return 0;
  return sizeof(double) * 3 * (size_t)T * (size_t)pf_chunks(m);
}

rpca_status rpca_prefilter(const float* X, int64_t m, int32_t T, double corr_min, int32_t window, float* Y,
                           int32_t* kept, int32_t* count, double* corr, void* scratch, void* stream) {
  return prefilter_impl(X, m, T, corr_min, window, Y, kept, count, corr, scratch, stream, false);
}

rpca_status rpca_prefilter_highpass(const float* X, int64_t m, int32_t T, double corr_min, int32_t window,
                                    float* Y, int32_t* kept, int32_t* count, double* corr, void* scratch,
                                    void* stream) {
  return prefilter_impl(X, m, T, corr_min, window, Y, kept, count, corr, scratch, stream, true);
}

}  // extern "C"
