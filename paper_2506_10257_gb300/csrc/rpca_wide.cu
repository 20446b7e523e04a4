// rpca_wide.cu -- host side of the wide / complex path: kernel tables.
#include <cuda_runtime.h>

#include "rpca_internal.h"
#include "rpca_wide.cuh"

namespace rpca {

template <int CW, bool CPLX>
WideKernels make_wide() {
  constexpr int TP = 8 * CW;
  WideKernels k;
  if constexpr (TP <= 128) {
    // Wbar and V resident in shared memory, 64-pixel tiles
    k.pass[PM_INIT] = (void*)pass_res_kernel<TP, PM_INIT, CPLX>;
    k.pass[PM_FUSED] = (void*)pass_res_kernel<TP, PM_FUSED, CPLX>;
    k.pass[PM_UPDATE] = (void*)pass_res_kernel<TP, PM_UPDATE, CPLX>;
    k.pass[PM_GRAM] = (void*)pass_res_kernel<TP, PM_GRAM, CPLX>;
    k.pass_smem = res_pass_smem_bytes(TP);
    k.tile = kRP;
    k.per_sm = res_blocks_per_sm(TP);
  } else {
    // Wbar and V streamed 32 rows at a time, 32-pixel tiles
    k.pass[PM_INIT] = (void*)pass_wide_kernel<CW, PM_INIT, CPLX>;
    k.pass[PM_FUSED] = (void*)pass_wide_kernel<CW, PM_FUSED, CPLX>;
    k.pass[PM_UPDATE] = (void*)pass_wide_kernel<CW, PM_UPDATE, CPLX>;
    k.pass[PM_GRAM] = (void*)pass_wide_kernel<CW, PM_GRAM, CPLX>;
    k.pass_smem = WideShape<CW>::smem;
    k.tile = kWP;
    k.per_sm = 1;
  }
  k.pass_threads = kWideThreads;
  k.eig = (void*)eig_wide_kernel;
  k.eig_threads = kEigWThreads;
  for (int i = 0; i < 4; ++i) {
    k.pass_tc[i] = nullptr;
    k.pass_tc_smem[i] = 0;
  }
  k.pass_tc_threads = kWtcThreads;
  // the tiled tensor-core pass: real windows of 33..128 frames, complex ones
  // of up to 64 frames (128 real columns; 16 frames and fewer padded to 64)
  constexpr int TPW = wtc_tp(TP);
  if constexpr ((CPLX || TP >= 64) && TPW <= 128) {
    k.pass_tc[RPCA_PREC_TF32X3] = (void*)pass_wtc_kernel<TPW, false, CPLX>;
    k.pass_tc_smem[RPCA_PREC_TF32X3] = WtcShape<TPW, false>::SMEM;
    k.pass_tc[RPCA_PREC_BF16X3] = (void*)pass_wtc_kernel<TPW, true, CPLX>;
    k.pass_tc_smem[RPCA_PREC_BF16X3] = WtcShape<TPW, true>::SMEM;
  }
  return k;
}

size_t wide_tc_img_bytes(int T, int precision) {
  const int TP = wtc_tp(T);
  if (TP > 128) return 0;
  if (precision == RPCA_PREC_TF32X3) return wtc_img_bytes(TP, false);
  if (precision == RPCA_PREC_BF16X3) return wtc_img_bytes(TP, true);
  return 0;
}

void wide_launch_shape(int T, int* tile, int* per_sm) {
  const int TP = (T + 31) / 32 * 32;
  *tile = TP <= 128 ? kRP : kWP;
  *per_sm = TP <= 128 ? res_blocks_per_sm(TP) : 1;
}

template <bool CPLX>
WideKernels pick_wide(int TP) {
  switch (TP) {
    case 32: return make_wide<4, CPLX>();
    case 64: return make_wide<8, CPLX>();
    case 96: return make_wide<12, CPLX>();
    case 128: return make_wide<16, CPLX>();
    case 160: return make_wide<20, CPLX>();
    case 192: return make_wide<24, CPLX>();
    default: return make_wide<28, CPLX>();
  }
}

bool wide_kernels(int T, bool cplx, bool force, WideKernels* out) {
  if (T > kMaxTW || T < 1) return false;
  if (!cplx && T <= kMaxT && !force) return false;
  if (cplx && (T & 1)) return false;
  const int TP = (T + 31) / 32 * 32;
  *out = cplx ? pick_wide<true>(TP) : pick_wide<false>(TP);
  out->eig_smem = eig_wide_smem(T, kVRows);
  if (cudaFuncSetAttribute(out->eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->eig_smem) != cudaSuccess)
    return false;
  for (int i = 0; i < 4; ++i)
    if (cudaFuncSetAttribute(out->pass[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->pass_smem) !=
        cudaSuccess)
      return false;
  for (int i = 0; i < 4; ++i)
    if (out->pass_tc[i] && cudaFuncSetAttribute(out->pass_tc[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)out->pass_tc_smem[i]) != cudaSuccess)
      return false;
  return true;
}

}  // namespace rpca
