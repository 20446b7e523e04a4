// rpca_batch_tc.cu -- the batched persistent kernel for windows whose two
// dense contractions run on the tensor cores (TF32x3 or BF16x3, FP32
// accumulation in TMEM): the same lanes, publication counters, paired slots
// and bounded waits as the FP32 batch kernel (rpca_batch.cuh), with the
// fused pass of every iteration taken by pass_tc_body.  The initial pass over
// X and the eigen-steps are the FP32 batch kernel's.  Kept in its own
// translation unit so it compiles in parallel with the rest of the library.
#include <cuda_runtime.h>

#include "rpca_kernels.cuh"
#include "rpca_internal.h"

namespace rpca {
#include "rpca_batch.cuh"

// TMEM columns each CTA of a tensor-core batch holds for the whole launch
// (Q and Z~ of the two warpgroups at up to 32 frames).
constexpr uint32_t kBatchTmemCols = 128;

// The CTA's TMEM allocation (written by warp 0 at the start of the launch).
__shared__ uint32_t g_batch_tmem;

// The bodies are called, not inlined, so that each compiles once for both
// lane runners (the paired and the sequential one), which keeps the build short.
template <int TB, bool BF16>
__device__ __noinline__ bool tc_pass_call(Bufs b, bool init, int lc, int nc, unsigned char* dsm) {
  if (init) return pass_body<TB, PM_INIT>(b, lc, nc, dsm);
  return pass_tc_body<TB, (TB <= 16 ? 16 : 32), BF16, true>(b, lc, nc, dsm, g_batch_tmem);
}
template <int TB>
__device__ __noinline__ void tc_eig_call(Bufs b, int flags, unsigned char* dsm) {
  NarrowBody<TB>::eig(b, flags, dsm, 0);
}

template <int TB, bool BF16>
struct TcBody {
  static_assert(4 * (TB <= 16 ? 16 : 32) <= (int)kBatchTmemCols, "TMEM columns");
  static __device__ bool pass(Bufs b, bool init, int lc, int nc, unsigned char* dsm) {
    return tc_pass_call<TB, BF16>(b, init, lc, nc, dsm);
  }
  static __device__ void eig(Bufs b, int flags, unsigned char* dsm, int) { tc_eig_call<TB>(b, flags, dsm); }
};

template <int TBMAX, bool BF16>
struct TcDisp {
  static __device__ bool pass(WinDesc& wd, bool init, int lc, int nc, unsigned char* dsm) {
    switch (wd.TB) {
      case 8: return TcBody<8, BF16>::pass(wd.b, init, lc, nc, dsm);
      case 12: return TcBody<12, BF16>::pass(wd.b, init, lc, nc, dsm);
      case 16: return TcBody<16, BF16>::pass(wd.b, init, lc, nc, dsm);
      case 20: return TcBody<20, BF16>::pass(wd.b, init, lc, nc, dsm);
      case 24: if constexpr (TBMAX >= 24) return TcBody<24, BF16>::pass(wd.b, init, lc, nc, dsm); break;
      case 32: if constexpr (TBMAX >= 32) return TcBody<32, BF16>::pass(wd.b, init, lc, nc, dsm); break;
      default: break;
    }
    return false;
  }
  static __device__ void eig(WinDesc& wd, int flags, unsigned char* dsm, int vrows) {
    switch (wd.TB) {
      case 8: TcBody<8, BF16>::eig(wd.b, flags, dsm, vrows); break;
      case 12: TcBody<12, BF16>::eig(wd.b, flags, dsm, vrows); break;
      case 16: TcBody<16, BF16>::eig(wd.b, flags, dsm, vrows); break;
      case 20: TcBody<20, BF16>::eig(wd.b, flags, dsm, vrows); break;
      case 24: if constexpr (TBMAX >= 24) TcBody<24, BF16>::eig(wd.b, flags, dsm, vrows); break;
      case 32: if constexpr (TBMAX >= 32) TcBody<32, BF16>::eig(wd.b, flags, dsm, vrows); break;
      default: break;
    }
  }
};

template <int TB, bool BF16>
__host__ __device__ constexpr size_t batch_tc_smem_tb() {
  return cmax(batch_smem_tb<TB>(), pass_tc_smem<TB, (TB <= 16 ? 16 : 32), BF16>());
}

template <int TBMAX, bool BF16>
__global__ void __launch_bounds__(kBatchThreads, 1) batch_kernel_tc(BatchDesc* bd) {
  extern __shared__ __align__(128) unsigned char batch_tc_dsm[];
  const int nl = bd->nlanes;
  int l = 0;
  while (l + 1 < nl && (int)blockIdx.x >= bd->lane[l + 1].cta0) ++l;
  const LaneDesc ld = bd->lane[l];
  const int lc = (int)blockIdx.x - ld.cta0;
  if (lc < 0 || lc >= ld.ncta) return;
  const unsigned long long limit = bd->spin_limit;
  // one TMEM allocation per CTA for the whole launch (one CTA per SM)
  if ((threadIdx.x >> 5) == 0) tmem_alloc(&g_batch_tmem, kBatchTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  run_lane<TcDisp<TBMAX, BF16>>(bd, ld, lc, batch_tc_dsm, limit, &bd->stop, 0, lane_is_paired(bd->paired, ld));
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(g_batch_tmem, kBatchTmemCols);
}

// One kernel per precision serves every frame bucket; its shared memory is
// the largest any bucket up to the batch's largest (tbmax) needs.
template <bool BF16>
size_t batch_tc_smem_upto(int tbmax) {
  size_t s = batch_tc_smem_tb<8, BF16>();
  if (tbmax >= 12) s = cmax(s, batch_tc_smem_tb<12, BF16>());
  if (tbmax >= 16) s = cmax(s, batch_tc_smem_tb<16, BF16>());
  if (tbmax >= 20) s = cmax(s, batch_tc_smem_tb<20, BF16>());
  if (tbmax >= 24) s = cmax(s, batch_tc_smem_tb<24, BF16>());
  if (tbmax >= 32) s = cmax(s, batch_tc_smem_tb<32, BF16>());
  return s;
}

void batch_tc_kernel_info(int tbmax, bool bf16, void** fn, size_t* smem) {
  *fn = bf16 ? (void*)batch_kernel_tc<32, true> : (void*)batch_kernel_tc<32, false>;
  *smem = bf16 ? batch_tc_smem_upto<true>(tbmax) : batch_tc_smem_upto<false>(tbmax);
}

}  // namespace rpca
