// rpca_noalloc.cu -- rotated-Gram entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc on their hot path: a real-time scanner
// pipeline that reserves all of its device memory once at start-up and must
// not block on the allocator (cudaMalloc can synchronise the device) while
// frames stream in, or a host process whose memory is owned by another
// framework's pool.  rpca_gram_noalloc computes the same Gram as rpca_gram
// with its scratch (partial Grams, reduction counters, control block) in a
// fixed array compiled into this library instead of allocated memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/rpca.h"

// The kernels get internal linkage in this translation unit so the library's
// other unit can define the same (non-template) kernels.
namespace {
#include "rpca_kernels.cuh"
}  // namespace

namespace {

using namespace rpca;

// Maximum CTAs whose partial Grams fit in the scratch array.
constexpr int kNaMaxGrid = 512;
constexpr int kNaMaxGroups = (kNaMaxGrid + kGroup - 1) / kGroup;

constexpr size_t na_align(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kNaCtrl = 0;
constexpr size_t kNaEig = na_align(kNaCtrl + sizeof(Ctrl));
constexpr size_t kNaRed = na_align(kNaEig + sizeof(EigState));
constexpr size_t kNaJob = na_align(kNaRed + sizeof(RedState));
constexpr size_t kNaHeader = na_align(kNaJob + sizeof(Job));      // zeroed by every call
constexpr size_t kNaGram = kNaHeader;
constexpr size_t kNaGroup = na_align(kNaGram + sizeof(float) * kNaMaxGrid * kMaxT * kMaxT);
constexpr size_t kNaScal = na_align(kNaGroup + sizeof(float2) * kNaMaxGroups * kMaxT * kMaxT);
constexpr size_t kNaGscal = na_align(kNaScal + sizeof(double) * 2 * kNaMaxGrid);
constexpr size_t kNaBytes = na_align(kNaGscal + sizeof(double) * 2 * kNaMaxGroups);  // about 2.4 MB

// The scratch: one copy per GPU that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_rpca_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
void* g_na_ptr[kNaMaxDevices];   // device address of the scratch, per device ...
void* g_na_ctx[kNaMaxDevices];   // ... and the context it was looked up in

// The calling thread's current CUDA context (driver cuCtxGetCurrent, looked
// up once through the runtime), or NULL when it cannot be had.
void* current_context() {
  typedef int (*CtxGetCurrent)(void**);
  static CtxGetCurrent fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrent)f;
  }
  void* ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}

// Device address of the scratch on the current device: looked up the first
// time a device is used, and again whenever the device's current context is
// another one than at the last lookup (after cudaDeviceReset the primary
// context, and with it the array's address, is new).
cudaError_t na_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_na_mu);
  void* ctx = current_context();
  if (!g_na_ptr[dev] || !ctx || ctx != g_na_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_rpca_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = p;
    g_na_ctx[dev] = current_context();  // (the lookup makes the primary context current)
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

// Job, control block and basis V (row-major T x T, NULL = identity) for one Gram.
__global__ void na_setup_kernel(Bufs b, const float* X, const float* V, int T) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    b.job->X = X;
    b.ctrl->k = 0;
    b.ctrl->done = 0;
    b.ctrl->f_inv_mu = 1.f;
    b.red->t_start = ~0ull;
  }
  for (int i = tid; i < kMaxT * kMaxT; i += blockDim.x) {
    const int r = i / kMaxT, c = i % kMaxT;
    float v = 0.f;
    if (r < T && c < T) v = V ? V[r * T + c] : (r == c ? 1.f : 0.f);
    b.eig->V32[i] = v;
  }
}

// G (row-major T x T, float64) from the reduced Gram.
__global__ void na_store_kernel(Bufs b, double* G, int T) {
  for (int i = threadIdx.x; i < T * T; i += blockDim.x) G[i] = b.red->G[(i / T) * kMaxT + i % T];
}

void* na_pass_fn(int T) {
  if (T <= 8) return (void*)pass_kernel<8, PM_GRAM>;
  if (T <= 12) return (void*)pass_kernel<12, PM_GRAM>;
  if (T <= 16) return (void*)pass_kernel<16, PM_GRAM>;
  if (T <= 20) return (void*)pass_kernel<20, PM_GRAM>;
  if (T <= 24) return (void*)pass_kernel<24, PM_GRAM>;
  return (void*)pass_kernel<32, PM_GRAM>;
}

size_t na_pass_smem(int T) {
  if (T <= 8) return pass_simt_smem<8>();
  if (T <= 12) return pass_simt_smem<12>();
  if (T <= 16) return pass_simt_smem<16>();
  if (T <= 20) return pass_simt_smem<20>();
  if (T <= 24) return pass_simt_smem<24>();
  return pass_simt_smem<32>();
}

rpca_status na_status(cudaError_t e) {
  if (e == cudaSuccess) return RPCA_OK;
  return RPCA_ERR_CUDA;
}

}  // namespace

extern "C" rpca_status rpca_gram_noalloc(const float* X, int64_t m, int32_t T, const float* V, double* G,
                                         void* stream) {
  if (!X || !G || m < 1 || T < 1) return RPCA_ERR_ARG;
  if (T > kMaxT) return RPCA_ERR_UNSUPPORTED;
  void* base = nullptr;
  cudaError_t e = na_scratch(&base);
  if (e != cudaSuccess) return na_status(e);
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return na_status(e);
  const int64_t ntiles = (m + kTile - 1) / kTile;
  const int64_t cap = (int64_t)kPassCtasPerSm * sms;
  int64_t grid = ntiles < cap ? ntiles : cap;
  if (grid > kNaMaxGrid) grid = kNaMaxGrid;
  if (grid < 1) grid = 1;

  char* s0 = (char*)base;
  Bufs b;
  memset(&b, 0, sizeof(b));
  b.ctrl = (Ctrl*)(s0 + kNaCtrl);
  b.eig = (EigState*)(s0 + kNaEig);
  b.red = (RedState*)(s0 + kNaRed);
  b.job = (Job*)(s0 + kNaJob);
  b.gram_part = (float*)(s0 + kNaGram);
  b.group_part = (float2*)(s0 + kNaGroup);
  b.scal_part = (double*)(s0 + kNaScal);
  b.gscal_part = (double*)(s0 + kNaGscal);
  b.m = m;
  b.T = T;
  b.grid = (int)grid;
  b.ngroups = (int)((grid + kGroup - 1) / kGroup);
  b.finalize = 1;

  cudaStream_t s = (cudaStream_t)stream;
  // The array keeps the previous call's contents: clear the control block and
  // the reduction counters, which must start at zero.
  e = cudaMemsetAsync(s0, 0, kNaHeader, s);
  void* a_setup[] = {&b, (void*)&X, (void*)&V, &T};
  if (e == cudaSuccess) e = cudaLaunchKernel((void*)na_setup_kernel, dim3(1), dim3(256), a_setup, 0, s);
  void* a_pass[] = {&b};
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(na_pass_fn(T), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)na_pass_smem(T));
  if (e == cudaSuccess)
    e = cudaLaunchKernel(na_pass_fn(T), dim3((unsigned)grid), dim3(kPassThreads), a_pass, na_pass_smem(T), s);
  void* a_store[] = {&b, &G, &T};
  if (e == cudaSuccess) e = cudaLaunchKernel((void*)na_store_kernel, dim3(1), dim3(256), a_store, 0, s);
  return na_status(e);
}
