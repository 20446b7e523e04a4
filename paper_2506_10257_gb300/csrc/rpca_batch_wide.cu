// rpca_batch_wide.cu -- the batched persistent kernel for batches that hold a
// wide (T > 32) or complex window: every window of such a batch runs the tiled
// pass and eigen-step bodies (rpca_wide.cuh) under the same lane schedule,
// publication counters and bounded waits as the narrow batch kernel
// (rpca_batch.cuh).  Kept in its own translation unit so it compiles in
// parallel with the rest of the library.
#include <cuda_runtime.h>

#include "rpca_kernels.cuh"
#include "rpca_internal.h"
#include "rpca_wide.cuh"

namespace rpca {
#include "rpca_batch.cuh"

// The tiled bodies are called, not inlined, into the one kernel that serves
// every column count: each compiles once, which keeps the build short.
template <int CW, int MODE, bool CPLX>
__device__ __noinline__ bool wide_pass_call(Bufs b, int lc, int nc, float* f) {
  return pass_wide_body<CW, MODE, CPLX>(b, lc, nc, f);
}
__device__ __noinline__ void wide_eig_call(Bufs b, int flags, float* f, int vrows) {
  eig_wide_body(b, flags, 0, 0, f, vrows);
}

template <int CW, bool CPLX>
struct WideBody {
  static __device__ bool pass(Bufs b, bool init, int lc, int nc, unsigned char* dsm) {
    float* f = reinterpret_cast<float*>(dsm);
    return init ? wide_pass_call<CW, PM_INIT, CPLX>(b, lc, nc, f) : wide_pass_call<CW, PM_FUSED, CPLX>(b, lc, nc, f);
  }
  static __device__ void eig(Bufs b, int flags, unsigned char* dsm, int vrows) {
    wide_eig_call(b, flags, reinterpret_cast<float*>(dsm), vrows);
  }
};

// The tiled steps of a window by its columns per warp (TB of the descriptor).
template <bool CPLX>
struct WideDisp {
  static __device__ bool pass(WinDesc& wd, bool init, int lc, int nc, unsigned char* dsm) {
    switch (wd.TB) {
      case 4: return WideBody<4, CPLX>::pass(wd.b, init, lc, nc, dsm);
      case 8: return WideBody<8, CPLX>::pass(wd.b, init, lc, nc, dsm);
      case 12: return WideBody<12, CPLX>::pass(wd.b, init, lc, nc, dsm);
      case 16: return WideBody<16, CPLX>::pass(wd.b, init, lc, nc, dsm);
      case 20: return WideBody<20, CPLX>::pass(wd.b, init, lc, nc, dsm);
      case 24: return WideBody<24, CPLX>::pass(wd.b, init, lc, nc, dsm);
      case 28: return WideBody<28, CPLX>::pass(wd.b, init, lc, nc, dsm);
      default: return false;
    }
  }
  static __device__ void eig(WinDesc& wd, int flags, unsigned char* dsm, int vrows) {
    wide_eig_call(wd.b, flags, reinterpret_cast<float*>(dsm), vrows);
  }
};

// Batches holding a wide or complex window: every window runs the tiled
// bodies (TB of a window = its columns per warp, CW).
template <bool CPLX>
__global__ void __launch_bounds__(kBatchThreads, 1) batch_kernel_wide(BatchDesc* bd) {
  extern __shared__ __align__(16) unsigned char batch_dsm[];
  const int nl = bd->nlanes;
  int l = 0;
  while (l + 1 < nl && (int)blockIdx.x >= bd->lane[l + 1].cta0) ++l;
  const LaneDesc ld = bd->lane[l];
  const int lc = (int)blockIdx.x - ld.cta0;
  if (lc < 0 || lc >= ld.ncta) return;
  const unsigned long long limit = bd->spin_limit;
  const int vrows = bd->vrows;
  run_lane<WideDisp<CPLX>>(bd, ld, lc, batch_dsm, limit, &bd->stop, vrows, lane_is_paired(bd->paired, ld));
}

void* batch_wide_kernel_fn(bool cplx) {
  return cplx ? (void*)batch_kernel_wide<true> : (void*)batch_kernel_wide<false>;
}

}  // namespace rpca
