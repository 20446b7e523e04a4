// rpca_wide.cu -- host side of the wide / complex path: kernel tables.
#include <cuda_runtime.h>

#include "rpca_internal.h"
#include "rpca_wide.cuh"

namespace rpca {

template <int CW, bool CPLX>
WideKernels make_wide() {
  WideKernels k;
  k.pass[PM_INIT] = (void*)pass_wide_kernel<CW, PM_INIT, CPLX>;
  k.pass[PM_FUSED] = (void*)pass_wide_kernel<CW, PM_FUSED, CPLX>;
  k.pass[PM_UPDATE] = (void*)pass_wide_kernel<CW, PM_UPDATE, CPLX>;
  k.pass[PM_GRAM] = (void*)pass_wide_kernel<CW, PM_GRAM, CPLX>;
  k.pass_smem = WideShape<CW>::smem;
  k.pass_threads = kWideThreads;
  k.tile = kWP;
  k.eig = (void*)eig_wide_kernel;
  k.eig_threads = kEigWThreads;
  return k;
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
  return true;
}

}  // namespace rpca
